// Tensor-core GEMM with fused epilogues (tcgen05, sm_103a), used by the surrogate MLP:
//   C[M][N] = A[M][K] * W[N][K]^T, BF16 operands, FP32 accumulate in TMEM
// (the kernel also supports the BF16 hi/lo split, products = 3: Ahi*Whi + Alo*Whi +
// Ahi*Wlo; the batched demag product uses the persistent grouped kernel in
// bpm_gemm_grouped.cu).
//
// One CTA computes a 128 x 256 output tile.  Warp 0 (one elected lane) streams the
// k-blocks (64 BF16 = one 128-byte swizzle atom) of every operand tile with TMA into a
// ring of shared-memory stages, warp 1 (one elected lane) issues the tcgen05.mma
// instructions into a 128-lane x 256-column TMEM accumulator, and after the last
// k-block all four warps read the accumulator back with tcgen05.ld and store it.
// Each stage holds Ahi, Alo, Whi, Wlo for one k-block, so the three products of a
// k-block share the staged tiles.  Every mbarrier wait is bounded; on timeout the
// kernel records an error flag, drains its own copies and MMAs, frees TMEM and exits.
#include <cuda.h>

#include "bpm_tc_ptx.cuh"

namespace bpm {

namespace {

using namespace tc;

// warp 0 issues the TMA loads and warp 1 the MMAs; all eight warps run the epilogue, warp w
// on TMEM lane quarter w % 4 (rows) and column half w / 4
constexpr int kThreads = 256;

// The forward layers of the MLP (bias+GELU and output epilogues) have K <= 256, at most four
// k-blocks: two stages keep their ring full and halve the shared memory, so that two CTAs share
// an SM and one CTA's epilogue runs beside the other's MMAs.  The other GEMMs (K = batch rows)
// keep the deep ring.
// The forward layers launch 128-wide column tiles: at 64 KB of ring a CTA, three CTAs (24 warps)
// share an SM for the GELU epilogue, which bounds these layers.
template <int P, int TN, int EPI>
struct Cfg {
    static constexpr int W_TILE = Tile<TN>::W_TILE;
    static constexpr int stage_bytes = (P == 3 ? 2 : 1) * (A_TILE + W_TILE);
    static constexpr bool forward_layer = EPI == 1 || EPI == 2;   // TC_EPI_BIAS_GELU, TC_EPI_BIAS_OUT
    static constexpr int stages = forward_layer ? 2 : (192 * 1024) / stage_bytes;   // 2 .. 6
    static constexpr int smem = stages * stage_bytes + 1024 /*align*/ + 256 /*barriers*/;
};

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Epilogue of one thread: row `row`, 32 accumulator columns starting at `col`.
template <int EPI>
__device__ __forceinline__ void epilogue32(const TcEpilogue& e, int M, int N, int row, int col, const uint32_t (&r)[32],
                                           float (&colsum)[32]) {
    const bool rok = row < M && row < e.rows_valid;
    if (EPI == TC_EPI_STORE) {
        if (!rok || col >= N) return;
        if (e.cols_valid >= N && (e.ldc % 4) == 0) {
            float4* dst = reinterpret_cast<float4*>(e.C + (size_t)row * e.ldc + col);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (col + 4 * q < N)
                    dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                         __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        } else {
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (col + q < e.cols_valid) e.C[(size_t)row * e.ldc + col + q] = __uint_as_float(r[q]);
        }
    } else if (EPI == TC_EPI_BIAS_GELU) {
        // z = acc + b; keep z (for the backward pass, optional) and h = GELU(z) row-major and,
        // optionally, transposed.  N is a multiple of 32 and the rows of H are 16-byte aligned,
        // so the 32 columns of h go out as four 16-byte stores.
        if (col >= N || row >= M) return;
        uint32_t hp[16];
#pragma unroll
        for (int q = 0; q < 32; q += 2) {
            float h2[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int c = col + q + u;
                const float z = __uint_as_float(r[q + u]) + (c < e.cols_valid ? e.bias[c] : 0.f);
                // rows past the valid batch are written as zeros so that no stale value travels on
                h2[u] = (rok && c < e.cols_valid) ? gelu(z) : 0.f;
                if (e.C && rok) e.C[(size_t)row * e.ldc + c] = z;
                if (e.HT) e.HT[(size_t)c * e.ldht + row] = __float2bfloat16_rn(h2[u]);
            }
            const __nv_bfloat162 pk = __floats2bfloat162_rn(h2[0], h2[1]);
            hp[q / 2] = *reinterpret_cast<const uint32_t*>(&pk);
        }
        uint4* dst = reinterpret_cast<uint4*>(e.H + (size_t)row * e.ldh + col);
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[v] = make_uint4(hp[4 * v], hp[4 * v + 1], hp[4 * v + 2], hp[4 * v + 3]);
    } else if (EPI == TC_EPI_BIAS_OUT) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int c = col + q;
            if (!rok || c >= e.cols_valid) break;
            const float z = __uint_as_float(r[q]) + e.bias[c];
            e.C[(size_t)row * e.ldc + c] = e.sigmoid ? 1.f / (1.f + expf(-z)) : z;
        }
    } else if (EPI == TC_EPI_GELU_BWD) {
        // dz = dh * GELU'(z) in both layouts, plus per-column sums for the bias gradient
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int c = col + q;
            float dz = 0.f;
            if (rok && c < e.cols_valid) dz = __uint_as_float(r[q]) * gelu_grad(e.Zin[(size_t)row * e.ldz + c]);
            colsum[q] = dz;
            if (c < N) {
                if (row < M) e.H[(size_t)row * e.ldh + c] = __float2bfloat16_rn(dz);
                if (e.HT && row < M) e.HT[(size_t)c * e.ldht + row] = __float2bfloat16_rn(dz);
            }
        }
    }
}

template <int P, int EPI, int TN>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
              const __grid_constant__ CUtensorMap mWhi, const __grid_constant__ CUtensorMap mWlo, int M, int N, int K,
              const TcEpilogue e, int* err) {
    using CF = Cfg<P, TN, EPI>;
    constexpr int W_TILE = CF::W_TILE;
    constexpr int S = CF::stages;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;             // 1024 B alignment for the swizzle atoms
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bar0 = base + S * CF::stage_bytes;         // full[S], empty[S], done, tmem slot
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
    const uint32_t done_bar = bar0 + 8u * (2 * S);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + S * CF::stage_bytes + 8 * (2 * S + 1));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * TN, m0 = blockIdx.y * TM;
    const int nk = K / TK;
    {   // an earlier launch gave up: skip (decided once per CTA, so that no thread is left at a barrier)
        __shared__ int s_abort;
        if (threadIdx.x == 0) s_abort = *(volatile int*)err;
        __syncthreads();
        if (s_abort) return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    auto sAhi = [&](int s) { return base + s * CF::stage_bytes; };
    auto sWhi = [&](int s) { return base + s * CF::stage_bytes + A_TILE; };
    auto sAlo = [&](int s) { return base + s * CF::stage_bytes + A_TILE + W_TILE; };
    auto sWlo = [&](int s) { return base + s * CF::stage_bytes + 2 * A_TILE + W_TILE; };

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int issued = 0;
        bool ok = true;
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % S;
            if (kb >= S) ok = mbar_wait(empty_bar(s), ((kb / S) - 1) & 1, err, 1);
            if (!ok) break;
            mbar_expect_tx(full_bar(s), CF::stage_bytes);
            const int kc = kb * TK;
            tma_load_2d(sAhi(s), &mAhi, kc, m0, full_bar(s));
            tma_load_2d(sWhi(s), &mWhi, kc, n0, full_bar(s));
            if (P == 3) {
                tma_load_2d(sAlo(s), &mAlo, kc, m0, full_bar(s));
                tma_load_2d(sWlo(s), &mWlo, kc, n0, full_bar(s));
            }
            issued = kb + 1;
        }
        // drain: every stage armed so far must have landed before the CTA may exit
        for (int kb = (issued > S ? issued - S : 0); kb < issued; ++kb)
            mbar_drain(full_bar(kb % S), (kb / S) & 1, err, 2);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        bool ok = true;
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % S;
            ok = mbar_wait(full_bar(s), (kb / S) & 1, err, 3);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int k = 0; k < TK / 16; ++k) {
                const uint32_t koff = 32u * k;
                const uint64_t ahi = sw128_desc(sAhi(s) + koff), whi = sw128_desc(sWhi(s) + koff);
                mma_bf16<TN>(tmem, ahi, whi, (kb > 0 || k > 0) ? 1u : 0u);
                if (P == 3) {
                    const uint64_t alo = sw128_desc(sAlo(s) + koff), wlo = sw128_desc(sWlo(s) + koff);
                    mma_bf16<TN>(tmem, alo, whi, 1u);
                    mma_bf16<TN>(tmem, ahi, wlo, 1u);
                }
            }
            mma_commit(empty_bar(s));
        }
        mma_commit(done_bar);       // tracks every MMA issued above, also on the error path
    }
    __syncwarp();
    // ---------------- epilogue: TMEM -> registers -> global ----------------
    const bool have = mbar_drain(done_bar, 0, err, 4);   // also on the error path: MMAs land before TMEM is freed
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // tcgen05.ld is warp-collective: take the decision once per warp
    const int go = __shfl_sync(0xffffffffu, (have && *(volatile int*)err == 0) ? 1 : 0, 0);
    if (go) {
        const int quarter = warp & 3, half = warp >> 2;
        const int row = m0 + quarter * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
        for (int c = half * (TN / 2); c < (half + 1) * (TN / 2); c += 32) {
            uint32_t r[32];
            float colsum[32];
            tmem_ld32(lane_addr + (uint32_t)c, r);
            const int col = n0 + c;
            epilogue32<EPI>(e, M, N, row, col, r, colsum);
            if (EPI == TC_EPI_GELU_BWD && e.colsum && col < N) {
                // fixed-order warp sums -> one partial per (row block of 32, column)
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    float v = colsum[q];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == q && col + q < N)
                        e.colsum[(size_t)(blockIdx.y * 4 + quarter) * e.ldcs + col + q] = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
    }
}

template <int P, int EPI, int TN = 256>
int launch(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo,
           const __nv_bfloat16* Whi, const __nv_bfloat16* Wlo, const TcEpilogue& e, int* err) {
    static bool configured = false;
    if (!configured) {
        BPM_CK(cudaFuncSetAttribute(k_gemm_tc<P, EPI, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Cfg<P, TN, EPI>::smem));
        configured = true;
    }
    CUtensorMap mAhi, mAlo, mWhi, mWlo;
    BPM_TRY(make_bf16_tensor_map(&mAhi, Ahi, K, M, TM));
    BPM_TRY(make_bf16_tensor_map(&mWhi, Whi, K, N, TN));
    if (P == 3) {
        BPM_TRY(make_bf16_tensor_map(&mAlo, Alo, K, M, TM));
        BPM_TRY(make_bf16_tensor_map(&mWlo, Wlo, K, N, TN));
    } else {
        mAlo = mAhi;
        mWlo = mWhi;
    }
    dim3 grid((N + TN - 1) / TN, M / TM);
    k_gemm_tc<P, EPI, TN><<<grid, kThreads, Cfg<P, TN, EPI>::smem, s>>>(mAhi, mAlo, mWhi, mWlo, M, N, K, e, err);
    BPM_CK(cudaGetLastError());
    return BPM_OK;
}

}  // namespace

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

int make_bf16_tensor_map(CUtensorMap* map, const void* ptr, int inner, int rows, int box_rows, int box_inner) {
    if (box_inner != 64 && box_inner != 32) {
        set_error("TMA box depth must be 64 or 32 elements (got %d)", box_inner);
        return BPM_ERR_ARG;
    }
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return BPM_ERR_CUDA;
    }
    if ((reinterpret_cast<uintptr_t>(ptr) & 15u) || (inner % 8)) {
        set_error("TMA operand not 16-byte aligned (ptr %p, inner %d)", ptr, inner);
        return BPM_ERR_ARG;
    }
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
    // rows of box_inner BF16 elements: 128 B rows with the 128-byte swizzle, 64 B rows with the 64-byte one
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapSwizzle sw = box_inner == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return BPM_ERR_CUDA;
    }
    return BPM_OK;
}

int gemm_tc(cudaStream_t s, int epi, int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* W,
            const TcEpilogue& e, int* err_flag) {
    if (M % TM || K % TK || N % 16 || M <= 0 || N <= 0) {
        set_error("tensor-core GEMM needs M %% %d == 0, K %% %d == 0, N %% 16 == 0 (M=%d N=%d K=%d)", TM, TK, M, N, K);
        return BPM_ERR_ARG;
    }
    switch (epi) {
        case TC_EPI_STORE: return launch<1, TC_EPI_STORE>(s, M, N, K, A, A, W, W, e, err_flag);
        case TC_EPI_BIAS_GELU: return launch<1, TC_EPI_BIAS_GELU, 128>(s, M, N, K, A, A, W, W, e, err_flag);
        case TC_EPI_BIAS_OUT: return launch<1, TC_EPI_BIAS_OUT, 128>(s, M, N, K, A, A, W, W, e, err_flag);
        case TC_EPI_GELU_BWD: return launch<1, TC_EPI_GELU_BWD>(s, M, N, K, A, A, W, W, e, err_flag);
        default: set_error("unknown epilogue %d", epi); return BPM_ERR_ARG;
    }
}

}  // namespace bpm
