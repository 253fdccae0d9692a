// PTX wrappers shared by the tcgen05 GEMM kernels (sm_103a): mbarriers with
// bounded waits, TMA tile loads, shared-memory matrix descriptors, tcgen05.mma
// with BF16 operands, commits and TMEM loads.
#pragma once
#include <cuda.h>

#include "bpm_internal.cuh"

namespace bpm {
namespace tc {

constexpr int TM = 128, TK = 64;           // output rows per CTA; TK = one 128 B swizzle row of BF16
constexpr int A_TILE = TM * TK * 2;         // 16 KB
template <int TN>
struct Tile {
    static constexpr int W_TILE = TN * TK * 2;   // 32 KB (TN = 256) or 16 KB (TN = 128)
};
constexpr unsigned long long kWaitNs = 200000000ull;      // 200 ms per wait (a normal wait is < 0.1 ms)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// non-blocking test of a phase (try_wait may suspend the thread until the phase completes)
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// bounded wait: returns false (and raises the error flag) if the phase does not complete
// within kWaitNs, or -- unless heed_err is false -- as soon as another CTA has raised the
// flag.  Waits that guard the lifetime of shared memory or TMEM (copies or MMAs still in
// flight) pass heed_err = false, so that they end only when the work has landed or the
// time limit has passed.
// limit_ns bounds the waits of a kernel's normal progress (kWaitNs unless a caller shortens it
// to exercise the failure path); drains always take kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code, bool heed_err = true,
                                          unsigned long long limit_ns = kWaitNs) {
    if (limit_ns < kWaitNs) {
        // a shortened limit: non-blocking polls with the clock read after each, so that a
        // limit below the time the phase takes is sure to run out
        const unsigned long long t0 = global_ns();
        for (;;) {
            if (mbar_test_wait(bar, parity)) return true;
            if (global_ns() - t0 > limit_ns || (heed_err && *(volatile int*)err != 0)) break;
        }
        atomicExch(err, code);
        return false;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 256; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns || (heed_err && *(volatile int*)err != 0)) break;
    }
    atomicExch(err, code);
    return false;
}

// wait for work in flight (copies, MMAs) before shared memory or TMEM is given up
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity, int* err, int code) {
    return mbar_wait(bar, parity, err, code, false, kWaitNs);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: K-major operand tile written by TMA with 128 B swizzle
// (rows of 128 B, 8-row groups 1024 B apart); start address advances 32 B per K=16 slice
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);       // start address
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                        // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                        // 128 B swizzle
    return d;
}

// the same for 64 B rows with the 64-byte swizzle (8-row groups 512 B apart)
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);       // start address
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
    d |= (uint64_t)(512 >> 4) << 32;               // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                        // descriptor version for tcgen05
    d |= (uint64_t)4 << 61;                        // 64 B swizzle
    return d;
}

// instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major, M = 128, N = TN
template <int TN>
struct Idesc {
    static constexpr uint32_t value = (1u << 4)              // D = F32
                                      | (1u << 7)            // A = BF16
                                      | (1u << 10)           // B = BF16
                                      | ((uint32_t)(TN >> 3) << 17)
                                      | ((uint32_t)(TM >> 4) << 24);
};

// the descriptor for an MMA n columns wide (16 <= n <= TN, n % 16 == 0)
template <int TN>
__device__ __forceinline__ uint32_t idesc_n(int n) {
    return (Idesc<TN>::value & ~(0x3Fu << 17)) | ((uint32_t)(n >> 3) << 17);
}

// D[tmem] (+)= A[adesc] * B[bdesc]^T with a run-time instruction descriptor
__device__ __forceinline__ void mma_bf16_desc(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

template <int TN>
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(Idesc<TN>::value), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


}  // namespace tc
}  // namespace bpm
