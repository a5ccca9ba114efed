// tcgen05 / mbarrier building blocks of the tensor-core far-field kernels (inline PTX):
// shared-memory matrix and instruction descriptors for K-major TF32 operands without swizzle,
// the TF32 high/low split (both parts rounded to nearest), bounded mbarrier waits and the MMA /
// commit instructions.
#pragma once
#include <cstdint>

namespace lspr {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte stride between 16-byte
// column groups along K, sbo = byte stride between 8-row groups
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(lbo >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;
}

// nearest TF32 value of x (round to nearest, ties away from zero).  A split x = hi + lo with
// hi = tf32_rn(x) and lo = tf32_rn(x - hi) leaves |x - hi - lo| <= 2^-22 |x|, unbiased; the
// products hi*hi + hi*lo + lo*hi of two split operands then miss only lo*lo (<= 2^-22 relative)
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
struct TfPair {
    float4 hi, lo;
};
__device__ __forceinline__ TfPair tf32_split(const float4 v) {
    TfPair p;
    p.hi = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
    p.lo = make_float4(tf32_rn(v.x - p.hi.x), tf32_rn(v.y - p.hi.y), tf32_rn(v.z - p.hi.z), tf32_rn(v.w - p.hi.w));
    return p;
}


__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity; false: it ran out (the abort flag is
// raised) or another role raised the flag
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    if (bar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (uint32_t it = 1;; ++it) {
        if (bar_try(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort_flag) return false;
            if (now_ns() - t0 > 1000000000ull) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}


// instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, N and M
constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// every lane waits; the verdict is made uniform over the warp (the callers then take
// .sync.aligned steps or warp syncs together)
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    const bool ok = bar_wait(bar, parity, abort_flag);
    return __all_sync(0xffffffffu, ok);
}

// wait for a phase that completes by itself (copies or MMAs in flight), bounded, whatever
// the abort flag says
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = now_ns();
    while (!bar_try(bar, parity) && now_ns() - t0 < 1000000000ull) {
    }
}


}  // namespace tc
}  // namespace lspr
