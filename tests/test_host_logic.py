"""Host-side logic of the serving engine, without a GPU: the first-fit arena
that enforces the device-memory admission budget (csrc/gpz_arena.hpp),
checked against a brute-force occupancy map over random alloc / release
sequences."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_10305_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include "gpz_arena.hpp"

// Brute force: one flag per 256-byte unit.
struct Model {
    std::vector<int> owner;  // -1 free, else the allocation's offset / 256
    explicit Model(uint64_t units) : owner(units, -1) {}
    bool free_run(uint64_t at, uint64_t n) const {
        for (uint64_t k = 0; k < n; ++k) if (owner[at + k] != -1) return false;
        return true;
    }
    // lowest unit where n free units start, or -1
    int64_t first_fit(uint64_t n) const {
        for (uint64_t at = 0; at + n <= owner.size(); ++at) if (free_run(at, n)) return (int64_t)at;
        return -1;
    }
    uint64_t largest() const {
        uint64_t best = 0, run = 0;
        for (int o : owner) { run = o == -1 ? run + 1 : 0; if (run > best) best = run; }
        return best;
    }
};

int main() {
    const uint64_t units = 512, cap = units * 256;
    gpz::host::Arena a(cap + 100);  // capacity rounds down to a multiple of 256
    Model m(units);
    if (a.capacity() != cap) { std::printf("capacity %llu\n", (unsigned long long)a.capacity()); return 1; }
    std::vector<std::pair<uint64_t, uint64_t>> live;  // offset, units
    uint64_t x = 12345;
    auto rnd = [&]() { x = x * 6364136223846793005ull + 1442695040888963407ull; return x >> 33; };
    uint64_t peak = 0, used = 0;
    for (int step = 0; step < 20000; ++step) {
        const bool do_alloc = live.empty() || rnd() % 100 < 55;
        if (do_alloc) {
            const uint64_t bytes = 1 + rnd() % (40 * 256);
            const uint64_t n = (bytes + 255) / 256;
            uint64_t off = 0;
            if (a.fits(bytes) != (m.largest() >= n)) { std::printf("step %d: fits\n", step); return 1; }
            const bool ok = a.alloc(bytes, &off);
            const int64_t want = m.first_fit(n);
            if (ok != (want >= 0)) { std::printf("step %d: alloc %d, model %lld\n", step, ok, (long long)want); return 1; }
            if (!ok) continue;
            if (off % 256 || off / 256 != (uint64_t)want) { std::printf("step %d: offset %llu vs %lld\n", step, (unsigned long long)off, (long long)want * 256); return 1; }
            for (uint64_t k = 0; k < n; ++k) m.owner[off / 256 + k] = (int)(off / 256);
            live.push_back({off, n});
            used += n * 256;
        } else {
            const size_t i = rnd() % live.size();
            if (!a.release(live[i].first)) { std::printf("step %d: release failed\n", step); return 1; }
            for (uint64_t k = 0; k < live[i].second; ++k) m.owner[live[i].first / 256 + k] = -1;
            used -= live[i].second * 256;
            live.erase(live.begin() + i);
            if (a.release(12345 * 256 + 7)) { std::printf("released an unknown offset\n"); return 1; }
        }
        if (used > peak) peak = used;
        if (a.used_bytes() != used || a.peak_bytes() != peak || a.largest_free() != m.largest() * 256) {
            std::printf("step %d: accounting\n", step);
            return 1;
        }
    }
    for (auto& l : live) a.release(l.first);
    if (a.used_bytes() != 0 || a.free_ranges() != 1 || a.largest_free() != cap || a.live_ranges() != 0) {
        std::printf("no full coalescing: %zu ranges\n", a.free_ranges());
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_arena_first_fit_matches_brute_force(tmp_path):
    src = tmp_path / "arena_check.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "arena_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I" + CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
