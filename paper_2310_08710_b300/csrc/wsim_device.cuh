// Device helpers of the wsim kernels (sm_103a): compensated float32
// arithmetic, oriented-box geometry, and bounded mbarrier waits for the
// bulk (TMA) copies that stage road-edge segments in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "wsim_internal.h"

namespace wsim {

// ---------------------------------------------------------------------------
// Compensated (hi, lo) float32 pairs.  TwoSum (Knuth) returns the rounded sum
// and its exact rounding error; __fadd_rn keeps nvcc from fusing or
// reordering the error terms.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) + d, renormalised so that |lo| <= ulp(hi)/2.
__device__ __forceinline__ void comp_add(float& hi, float& lo, float d) {
    float s, e;
    two_sum(hi, d, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// cos and sin of (hi + lo) with lo tiny: first-order correction of the
// float32 values at hi (the neglected term is O(lo^2) < 1e-11).
__device__ __forceinline__ void comp_sincos(float hi, float lo, float& c, float& s) {
    float sh, ch;
    sincosf(hi, &sh, &ch);
    c = fmaf(-sh, lo, ch);
    s = fmaf(ch, lo, sh);
}

// Difference of two compensated values, rounded once: (ah + al) - (bh + bl).
__device__ __forceinline__ float comp_diff(float ah, float al, float bh, float bl) {
    return __fadd_rn(__fsub_rn(ah, bh), __fsub_rn(al, bl));
}

// ---------------------------------------------------------------------------
// SAT overlap depth of two oriented boxes (Sec. 3.4, collision): the minimum
// over the four edge normals of (rA + rB - |d . axis|).  With C = uA . uB
// and S = uA x uB the projected half extents reduce to hl|C| + hw|S| forms.
// Positive iff the boxes overlap.  (dx, dy) = centre of B minus centre of A.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sat_depth(float dx, float dy, float cA, float sA, float hlA, float hwA,
                                           float cB, float sB, float hlB, float hwB) {
    float C = fmaf(cA, cB, sA * sB);
    float S = fmaf(cA, sB, -sA * cB);
    float aC = fabsf(C), aS = fabsf(S);
    float pA = fabsf(fmaf(dx, cA, dy * sA));    // d . uA
    float qA = fabsf(fmaf(-dx, sA, dy * cA));   // d . nA
    float pB = fabsf(fmaf(dx, cB, dy * sB));    // d . uB
    float qB = fabsf(fmaf(-dx, sB, dy * cB));   // d . nB
    float o0 = hlA + fmaf(hlB, aC, hwB * aS) - pA;
    float o1 = hwA + fmaf(hlB, aS, hwB * aC) - qA;
    float o2 = hlB + fmaf(hlA, aC, hwA * aS) - pB;
    float o3 = hwB + fmaf(hlA, aS, hwA * aC) - qB;
    return fminf(fminf(o0, o1), fminf(o2, o3));
}

// ---------------------------------------------------------------------------
// Status word: the first error code recorded wins.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (TMA, non-tensor form).  Waits are bounded by the
// global timer; an expired wait returns false and the caller records
// WSIM_ETIMEOUT and leaves the scene.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of bar to complete, for at most limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

}  // namespace wsim
