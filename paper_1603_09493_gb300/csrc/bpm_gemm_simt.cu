// CUDA-core demag GEMMs: C[M][N] = A[M][K] * W[N][K]^T (both operands K-major).
//
// The FP32 instance is the plain (single-precision) form of the demag product
// H_d = N' (Ms m); the BF16x3 instance evaluates, on CUDA cores, the same three
// split products hi*hi + lo*hi + hi*lo that the tensor-core kernel computes,
// and serves to validate it.  128x128 output tile per CTA, 256 threads with an
// 8x8 register tile each, K staged through shared memory 8 at a time.
#include "bpm_internal.cuh"

namespace bpm {

namespace {

constexpr int BM = 128, BN = 128, BK = 8;

template <bool SPLIT>
__global__ void __launch_bounds__(256) k_gemm_nt(int M, int N, int K, const float* __restrict__ A, int lda,
                                                  const float* __restrict__ W, int ldw,
                                                  const __nv_bfloat16* __restrict__ Ahi,
                                                  const __nv_bfloat16* __restrict__ Alo,
                                                  const __nv_bfloat16* __restrict__ Whi,
                                                  const __nv_bfloat16* __restrict__ Wlo, int products,
                                                  float* __restrict__ C, int ldc) {
    __shared__ float As[BK][BM + 4], Ws[BK][BN + 4];
    __shared__ float Als[SPLIT ? BK : 1][SPLIT ? BM + 4 : 1], Wls[SPLIT ? BK : 1][SPLIT ? BN + 4 : 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[8][8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int p = 0; p < 8; ++p) acc[q][p] = 0.f;
    // loader: thread handles row lr (0..127) and k-half lk (0 or 4)
    const int lr = tid >> 1, lk = (tid & 1) * 4;
    for (int k0 = 0; k0 < K; k0 += BK) {
        int gm = m0 + lr, gn = n0 + lr;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int gk = k0 + lk + u;
            bool okk = gk < K;
            if (!SPLIT) {
                As[lk + u][lr] = (gm < M && okk) ? A[(size_t)gm * lda + gk] : 0.f;
                Ws[lk + u][lr] = (gn < N && okk) ? W[(size_t)gn * ldw + gk] : 0.f;
            } else {
                As[lk + u][lr] = (gm < M && okk) ? __bfloat162float(Ahi[(size_t)gm * lda + gk]) : 0.f;
                Als[lk + u][lr] = (gm < M && okk) ? __bfloat162float(Alo[(size_t)gm * lda + gk]) : 0.f;
                Ws[lk + u][lr] = (gn < N && okk) ? __bfloat162float(Whi[(size_t)gn * ldw + gk]) : 0.f;
                Wls[lk + u][lr] = (gn < N && okk) ? __bfloat162float(Wlo[(size_t)gn * ldw + gk]) : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[8], w[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = As[kk][ty + 16 * q];
#pragma unroll
            for (int p = 0; p < 8; ++p) w[p] = Ws[kk][tx + 16 * p];
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int p = 0; p < 8; ++p) acc[q][p] = fmaf(a[q], w[p], acc[q][p]);
            if (SPLIT && products > 1) {
                float al[8], wl[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) al[q] = Als[kk][ty + 16 * q];
#pragma unroll
                for (int p = 0; p < 8; ++p) wl[p] = Wls[kk][tx + 16 * p];
#pragma unroll
                for (int q = 0; q < 8; ++q)
#pragma unroll
                    for (int p = 0; p < 8; ++p) {
                        acc[q][p] = fmaf(al[q], w[p], acc[q][p]);
                        acc[q][p] = fmaf(a[q], wl[p], acc[q][p]);
                    }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        int gm = m0 + ty + 16 * q;
        if (gm >= M) continue;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            int gn = n0 + tx + 16 * p;
            if (gn < N) C[(size_t)gm * ldc + gn] = acc[q][p];
        }
    }
}

}  // namespace

int gemm_f32_nt(cudaStream_t s, int M, int N, int K, const float* A, int lda, const float* W, int ldw, float* C,
                int ldc) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm_nt<false><<<grid, 256, 0, s>>>(M, N, K, A, lda, W, ldw, nullptr, nullptr, nullptr, nullptr, 1, C, ldc);
    BPM_CK(cudaGetLastError());
    return BPM_OK;
}

int gemm_bf16x3_simt(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo,
                     const __nv_bfloat16* Whi, const __nv_bfloat16* Wlo, float* C, int products) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm_nt<true><<<grid, 256, 0, s>>>(M, N, K, nullptr, K, nullptr, K, Ahi, Alo, Whi, Wlo, products, C, N);
    BPM_CK(cudaGetLastError());
    return BPM_OK;
}

}  // namespace bpm
