// fmm_queue.cuh -- the device-side brick queue shared by the march kernels and
// the adjoint: a ring of (sequence << 32 | brick + 1) words, its head, tail
// and pending counters in the control block, and a time source for bounded
// waits.  A brick is in the ring at most once (its queued flag), so a ring of
// one slot per brick never overflows.  Every wait gives up after wait_ns of
// the control block (device time without progress): it sets ERR_SPIN and
// returns.
#pragma once

#include "fmm_internal.h"

namespace fmmgb {
namespace {

__device__ __forceinline__ unsigned long long device_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long vload(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }

// Push brick b (the caller has claimed queued[b] and counted it in pending).
__device__ __forceinline__ bool queue_push(Control *c, unsigned long long *q, unsigned long long cap,
                                           long long b)
{
    const unsigned long long t = atomicAdd(&c->q_tail, 1ull);
    const unsigned long long v = ((t & 0xffffffffull) << 32) | (unsigned long long)(b + 1);
    unsigned long long *slot = q + (t % cap);
    const unsigned long long t0 = device_ns(), lim = vload(&c->wait_ns);
    for (;;) {
        if (atomicCAS(slot, 0ull, v) == 0ull)
            return true;
        if (device_ns() - t0 > lim || (vload((const int *)&c->error) & ERR_SPIN))
            break;
        __nanosleep(32);
    }
    atomicOr(&c->error, ERR_SPIN);
    return false;
}

// Pop a brick: -1 when the restart is complete (or on a timeout).  Each
// caller takes a ticket from q_head and waits on its own slot, so idle warps
// poll distinct lines with a growing back-off instead of racing on the head.
// pending == 0 means that no push is in flight or to come, so a ticket whose
// slot is still empty then ends the caller's loop.  The time limit counts from
// the last push seen anywhere.
__device__ __forceinline__ long long queue_pop(Control *c, unsigned long long *q,
                                               unsigned long long cap)
{
    const unsigned long long h = atomicAdd(&c->q_head, 1ull);
    unsigned long long *slot = q + (h % cap);
    const unsigned long long want = h & 0xffffffffull;
    unsigned long long t0 = device_ns(), seen = vload(&c->q_tail);
    const unsigned long long lim = vload(&c->wait_ns);
    unsigned ns = 64;
    for (;;) {
        unsigned long long v = vload(slot);
        if (v != 0ull && (v >> 32) == want) {
            atomicExch(slot, 0ull);
            return (long long)(v & 0xffffffffull) - 1;
        }
        if (vload(&c->pending) == 0) {
            v = vload(slot);
            if (v != 0ull && (v >> 32) == want) {
                atomicExch(slot, 0ull);
                return (long long)(v & 0xffffffffull) - 1;
            }
            return -1;
        }
        if (vload(&c->error) & ERR_SPIN)
            return -1;
        const unsigned long long now = device_ns(), tail = vload(&c->q_tail);
        if (tail != seen) {
            seen = tail;
            t0 = now;
        } else if (now - t0 > lim) {
            break;
        }
        __nanosleep(ns);
        if (ns < 2048)
            ns <<= 1;
    }
    atomicOr(&c->error, ERR_SPIN);
    return -1;
}


}  // namespace
}  // namespace fmmgb
