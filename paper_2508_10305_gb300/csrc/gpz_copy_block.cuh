// gpz_copy_block.cuh -- the copy of a block from its 16-byte aligned
// temporary slot to its place in the stream (step 3 of Section 4.4's
// compaction), shared by the single-array and the batched compaction kernels.
#pragma once

#include "gpz_internal.cuh"

namespace gpz {

// One warp: len words from a 16-byte aligned slot to a word-aligned place
// in the stream.  The destination is cut into 16-byte units: a unit inside
// the block's words is written with one 16-byte store, assembled from the
// slot's 16-byte words k-1 and k (whole when the destination is aligned,
// else by a shuffle of the preceding lane's word); the first and last units,
// which the neighbouring blocks share, are written word by word.  Two units
// per lane are in flight; every slot read stays below the block's length.
__device__ __forceinline__ uint4 realign(uint4 prev, uint4 cur, uint32_t r) {
    switch (r) {
        case 1: return make_uint4(prev.w, cur.x, cur.y, cur.z);
        case 2: return make_uint4(prev.z, prev.w, cur.x, cur.y);
        case 3: return make_uint4(prev.y, prev.z, prev.w, cur.x);
        default: return cur;
    }
}

__device__ __forceinline__ void store_unit(uint32_t* dst_al, uint32_t u, uint4 v, uint32_t r, uint32_t len) {
    const int k0 = 4 * (int)u - (int)r;  // block word of the unit's first word
    uint4* d4 = reinterpret_cast<uint4*>(dst_al) + u;
    if (k0 >= 0 && k0 + 4 <= (int)len) {
        *d4 = v;
    } else {
        uint32_t* d = reinterpret_cast<uint32_t*>(d4);
        if (k0 >= 0 && k0 < (int)len) d[0] = v.x;
        if (k0 + 1 >= 0 && k0 + 1 < (int)len) d[1] = v.y;
        if (k0 + 2 >= 0 && k0 + 2 < (int)len) d[2] = v.z;
        if (k0 + 3 >= 0 && k0 + 3 < (int)len) d[3] = v.w;
    }
}

__device__ __forceinline__ void copy_block(const uint32_t* src, uint32_t* dst, uint32_t len, int lane) {
    const uint32_t r = (uint32_t)(reinterpret_cast<uintptr_t>(dst) >> 2) & 3u;  // words past a 16-byte boundary
    uint32_t* dst_al = dst - r;
    const uint32_t units = (len + r + 3u) >> 2;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    uint4 carry = zero;  // slot word u0 - 1 (lane 31's second word of the last round)
    for (uint32_t u0 = 0; u0 < units; u0 += 64) {
        const uint32_t ua = u0 + lane, ub = u0 + 32 + lane;
        const uint4 va = 4u * ua < len ? __ldcs(s4 + ua) : zero;
        const uint4 vb = 4u * ub < len ? __ldcs(s4 + ub) : zero;
        uint4 pa, pb;  // slot words ua - 1 and ub - 1
        pa.x = __shfl_up_sync(0xffffffffu, va.x, 1);
        pa.y = __shfl_up_sync(0xffffffffu, va.y, 1);
        pa.z = __shfl_up_sync(0xffffffffu, va.z, 1);
        pa.w = __shfl_up_sync(0xffffffffu, va.w, 1);
        pb.x = __shfl_up_sync(0xffffffffu, vb.x, 1);
        pb.y = __shfl_up_sync(0xffffffffu, vb.y, 1);
        pb.z = __shfl_up_sync(0xffffffffu, vb.z, 1);
        pb.w = __shfl_up_sync(0xffffffffu, vb.w, 1);
        const uint4 a31 = make_uint4(__shfl_sync(0xffffffffu, va.x, 31), __shfl_sync(0xffffffffu, va.y, 31),
                                     __shfl_sync(0xffffffffu, va.z, 31), __shfl_sync(0xffffffffu, va.w, 31));
        if (lane == 0) {
            pa = carry;
            pb = a31;
        }
        carry = make_uint4(__shfl_sync(0xffffffffu, vb.x, 31), __shfl_sync(0xffffffffu, vb.y, 31),
                           __shfl_sync(0xffffffffu, vb.z, 31), __shfl_sync(0xffffffffu, vb.w, 31));
        if (ua < units) store_unit(dst_al, ua, realign(pa, va, r), r, len);
        if (ub < units) store_unit(dst_al, ub, realign(pb, vb, r), r, len);
    }
}

}  // namespace gpz
