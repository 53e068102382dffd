// Persistent fused line compression with TMA prefetch.
//
// The plain kernel (one block per line) loads its line and only then
// computes, so an SM alternates between waiting on HBM and computing with the
// few lines its registers allow.  Here each block stays resident, walks the
// lines blockIdx.x, blockIdx.x + gridDim.x, ... and keeps the next line in
// flight while it computes the current one: a one-dimensional bulk TMA copy
// (cp.async.bulk, completion counted on an mbarrier) streams line i+1 into
// one of two shared-memory buffers while line i is transformed in the other.
// The same buffer then serves as the line's exchange buffer for the passes,
// so a block needs two line buffers of shared memory, not three.
//
// Waits are bounded: if a buffer's mbarrier does not complete within
// `wait_cycles` SM clocks the block records SAR status 5 (timeout) in
// *status, waits (bounded again) for any copy of its own still in flight,
// and returns.  No wait can hang the GPU.
//
// Why that exit is safe: a block must not end while a bulk copy it started
// can still write its shared memory.  Every copy this kernel starts reads a
// whole line that lies inside `in` (line < n_lines, 16-byte aligned, a
// multiple of 16 bytes) into this block's own shared memory, and its
// expect_tx byte count equals the copy's size.  Such a copy depends on no
// other block, thread or event: once issued it completes after one trip
// through the memory system (microseconds, against a bound of about a
// second).  A wait can therefore run out only on a copy that was never
// started (the injected fault below; `pending` stays false for it), and the
// exit's bounded wait on the copies that were started ends by their
// completion, never by its bound.  The block leaves through that path only
// after the pending copies' barriers have completed.
#pragma once

#include "line_engine.cuh"

namespace sar {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// order this thread's (and, after a barrier, the block's) generic-proxy
// shared-memory accesses before later async-proxy (TMA) accesses
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One elected thread: expect `bytes` on `bar` and start the bulk copy
// global -> shared.  src, dst 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_line_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with parity `parity`; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long wait_cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > wait_cycles) return false;
    }
    return true;
}

template <class SC>
struct PersistentLayout {
    // each line buffer: the padded exchange layout (>= N elements), rounded to 128 B
    static constexpr int BUF_ELEMS = ((SC::SMEM_ELEMS * 8 + 127) / 128) * 128 / 8;
    static constexpr int SMEM_BYTES = 2 * BUF_ELEMS * 8 + 2 * 8;  // two buffers + two mbarriers
};

// Test hook: when skip_line >= 0 the copy of that line is never started, so
// its wait must run out and the kernel must report a timeout.
template <class SC>
__global__ void __launch_bounds__(SC::T)
fused_persistent_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt,
                        const float2* tw, int* status, long long wait_cycles, int64_t skip_line) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using L = PersistentLayout<SC>;
    float2* bufs = reinterpret_cast<float2*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + 2 * L::BUF_ELEMS * 8);
    __shared__ int s_fail;
    const int t = threadIdx.x;
    const int64_t stride = gridDim.x;
    constexpr uint32_t kLineBytes = SC::N * 8;

    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_fail = 0;
    }
    __syncthreads();
    int64_t line = blockIdx.x;
    // thread 0 alone starts copies; pending[b]: a copy into buffer b was
    // started and its completion not yet observed
    bool pending[2] = {false, false};
    if (t == 0) {
        for (int b = 0; b < 2; ++b) {
            const int64_t l = line + b * stride;
            if (l < n_lines && l != skip_line) {
                tma_line_load(bufs + b * L::BUF_ELEMS, in + l * ld, kLineBytes, &bars[b]);
                pending[b] = true;
            }
        }
    }

    uint32_t parity[2] = {0u, 0u};
    for (int k = 0; line < n_lines; ++k, line += stride) {
        const int b = k & 1;
        float2* buf = bufs + b * L::BUF_ELEMS;
        if (mbar_wait_bounded(&bars[b], parity[b], wait_cycles))
            pending[b] = false;
        else
            s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        parity[b] ^= 1u;
        float2 v[SC::E];
        // pass-1 geometry from the linear copy: element lo + r*S1
#pragma unroll
        for (int s = 0; s < SC::E / SC::R1; ++s) {
            const int lo = t + SC::T * s;
#pragma unroll
            for (int r = 0; r < SC::R1; ++r) v[s * SC::R1 + r] = buf[lo + r * SC::S1];
        }
        __syncthreads();   // the linear copy is consumed before the exchanges reuse the buffer
        forward_passes<SC, 1>(v, buf, tw, t, 0);
        filter_multiply<SC>(filt, t, v);
        inverse_passes<SC, 1>(v, buf, tw, t, 0);
        __syncthreads();   // every read of this buffer is done: it may be refilled
        const int64_t next = line + 2 * stride;
        if (t == 0 && next < n_lines && next != skip_line) {
            fence_proxy_async_smem();
            tma_line_load(buf, in + next * ld, kLineBytes, &bars[b]);
            pending[b] = true;
        }
        global_store<SC, false>(out + line * ld, SC::N, t, v);
    }
    if (s_fail && t == 0) {
        atomicMax(status, 5);
        // let every copy this block started land before the block (and its
        // shared memory) goes away; bounded as well
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_wait_bounded(&bars[b], parity[b], wait_cycles);
    }
}

}  // namespace sar
