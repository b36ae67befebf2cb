// Bounded grid barrier of the cooperative kernels (shared by the translation
// units that launch them).
#pragma once

#include <cuda_runtime.h>

#include "ls_common.cuh"

namespace ls {
namespace {

constexpr long long kSpinLimit = 1LL << 24;   // ~1-2 s of polling with nanosleep

// ---------------------------------------------------------------------------
// bounded grid barrier (sense by generation counter); all CTAs must be
// co-resident (cooperative launch). On timeout the flag is raised and every
// CTA returns false.
// ---------------------------------------------------------------------------
__device__ bool group_barrier_n(DevStatus* st, unsigned int nblocks, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (nblocks <= 1) return true;
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &st->bar_gen;
        volatile int* vflag = &st->flag;
        unsigned int g = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(&st->bar_count, 1u);
        int ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == g) {
                if (*vflag != FLAG_OK) { ok = 0; break; }
                if (++it > limit) { atomicCAS(&st->flag, FLAG_OK, FLAG_TIMEOUT); ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (*vflag != FLAG_OK) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ bool group_barrier(DevStatus* st, unsigned int nblocks) { return group_barrier_n(st, nblocks, kSpinLimit); }

// Counting barrier: st->arrive only grows (zeroed before the launch), so the
// e-th barrier of nb CTAs waits for e * nb arrivals and needs neither a reset
// nor a generation word: one atomic and a polled load, where group_barrier
// takes a load, an atomic and, for the last CTA, two more atomics. The arrival
// is a release at GPU scope (it orders the CTA's writes, which the CTA barrier
// before it orders before thread 0's) and the poll an acquire, in place of two
// full fences. Bounded like group_barrier: on timeout, or when another CTA
// raised the flag, it returns false.
__device__ bool count_barrier(DevStatus* st, unsigned int target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&st->arrive) : "memory");
        volatile int* vflag = &st->flag;
        int ok = 1;
        long long it = 0;
        for (;;) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&st->arrive) : "memory");
            if (v >= target) break;
            if (*vflag != FLAG_OK) { ok = 0; break; }
            if (++it > kSpinLimit) { atomicCAS(&st->flag, FLAG_OK, FLAG_TIMEOUT); ok = 0; break; }
            __nanosleep(20);
        }
        if (*vflag != FLAG_OK) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace
}  // namespace ls
