/*
 * gpz_test.h -- failure-injection hooks of libgpz, for tests only.
 *
 * The paper has no counterpart: these entry points exist so that tests can
 * drive the library's failure paths -- a device-side wait that runs out, a
 * device allocation that fails -- without faulting or hanging a GPU.  The
 * waits in question are the look-backs of the compaction scan (Section 4.4,
 * step 2: a CTA waits for its predecessor tile's published prefix) and of
 * fused compaction (a block waits for its predecessors' published sizes).
 * Every such wait is bounded in the product kernels (about a second of SM
 * clock for the scans, about 60 us for the block look-back); these hooks run
 * the same kernels with a predecessor that never publishes and a short limit,
 * so that the wait runs out at once.  No hook enqueues anything that can
 * fault, and none changes the behaviour of other calls except
 * gpz_test_fail_next_allocations, which is process-wide by design.
 */
#ifndef GPZ_TEST_H
#define GPZ_TEST_H

#include <stdint.h>

#include "gpz.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Make the next `count` device allocations of the library fail as if the
 * device were out of memory: the workspace allocations of calls given
 * d_ws = NULL (which then return GPZ_ERR_OOM and enqueue nothing), batch plan
 * creation (GPZ_ERR_OOM) and the serving engine's arena (GPZ_ERR_OOM).
 * count = 0 disarms.  Returns how many failures were still armed before the
 * call.  Process-wide: every thread's calls draw on the same count. */
int gpz_test_fail_next_allocations(int count);

/* Device workspace in bytes for gpz_test_scan_timeout (256-byte aligned). */
uint64_t gpz_test_scan_workspace_size(void);

/* Run the compaction's look-back scan (Section 4.4, step 2) -- the
 * single-array kernel (batched = 0) or the batched one (batched = 1) -- over
 * 2 * 4096 + 1 block sizes, three tiles, with tile 0 never processed: the
 * CTAs take tiles 1 and 2, and tile 1's wait for tile 0's prefix runs out
 * after wait_cycles SM cycles (1..2^24).  The kernel then records
 * GPZ_ERR_TIMEOUT in the status word and finishes as if the missing prefix
 * were 0.  d_ws: gpz_test_scan_workspace_size() bytes.  Synchronises `stream`
 * and returns the device-side status (GPZ_ERR_TIMEOUT when the wait ran out,
 * as it must), or an argument / CUDA error. */
gpz_status gpz_test_scan_timeout(int batched, uint32_t wait_cycles, void* d_ws, uint64_t ws_size, void* stream);

/* The look-back over blocks of fused compaction, run by one warp for block
 * `block` (1..4096) while no block before it has published its size: the
 * wait for block-1 runs out after wait_cycles SM cycles (1..2^24) and the
 * block is reported unplaced (it would go through its temporary slot and
 * the copy kernel, which is not an error).  d_ws: at least
 * 8 * (block + 1) bytes, 256-byte aligned (the per-block states, cleared by
 * the call).  Synchronises `stream`; *h_placed receives 1 if the look-back
 * returned an offset, 0 if it gave up.  Returns GPZ_OK or an argument / CUDA
 * error. */
gpz_status gpz_test_block_lookback_timeout(uint32_t block, uint32_t wait_cycles, void* d_ws, uint64_t ws_size,
                                           int* h_placed, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GPZ_TEST_H */
