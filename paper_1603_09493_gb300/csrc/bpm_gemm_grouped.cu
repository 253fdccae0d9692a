// Persistent, grouped demag GEMM on the tensor cores (tcgen05, sm_103a).
//
// One launch computes, for every mesh group g of a batch (uneven mesh sizes),
//   C_g[M_g][N_g] = sum of the BF16 split products of A_g[M_g][K_g] and W_g[N_g][K_g]^T
// (3 products hi*hi + lo*hi + hi*lo, or 1), FP32 accumulate in TMEM.  The
// 128 x TN output tiles of all groups form one list; each CTA (one per SM)
// walks it with a stride of the grid size.  Within a group the tiles run
// M-major or N-major (chosen per group), so that a wave of CTAs shares the
// larger operand's rows in L2 and it is read from HBM once.  Warp roles:
//   warp 0  one lane streams the k-blocks of every tile with TMA into a ring of
//           shared-memory stages (the ring runs across tile boundaries);
//   warp 1  allocates two TMEM accumulators; one lane issues the MMAs, tile i
//           into accumulator i % 2;
//   warps 2-5  read an accumulator back (tcgen05.ld) and store it, while the
//           MMAs of the next tile run into the other accumulator.
// Per-group tensor maps live in a device array (64-byte aligned entries).
// Every wait is bounded; on timeout the kernel raises the error flag, drains
// its copies and MMAs, frees TMEM and exits, and later launches return at once.
// The waits of normal progress take the launch's limit (wait_ns); the drains
// always take the fixed limit, so that copies and MMAs land before shared
// memory or TMEM is given up.
#include <cstring>

#include "bpm_tc_ptx.cuh"

namespace bpm {

namespace {

using namespace tc;

constexpr int kGThreads = 192;

// KB: K depth of a stage (64: 128 B rows, 128-byte swizzle; 32: 64 B rows, 64-byte swizzle)
template <int P, int TN, int KB>
struct GCfg {
    static constexpr int A_BYTES = TM * KB * 2;
    static constexpr int W_BYTES = TN * KB * 2;
    static constexpr int stage_bytes = (P == 3 ? 2 : 1) * (A_BYTES + W_BYTES);
    static constexpr int stages = (192 * 1024) / stage_bytes;
    static constexpr int smem = stages * stage_bytes + 1024 + 256;
    static_assert(8 * (2 * stages + 5) + 4 <= 256, "barrier area");
};

template <int KB>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr) {
    return KB == 64 ? sw128_desc(addr) : sw64_desc(addr);
}

__device__ __forceinline__ int find_group(const GemmGroupDev* __restrict__ G, int ng, int t) {
    int g = 0;
    while (g + 1 < ng && t >= G[g + 1].tile_begin) ++g;
    return g;
}

// output tile lt of group gg -> first row (M) and column (N)
template <int TN>
__device__ __forceinline__ void tile_origin(const GemmGroupDev& gg, int lt, int& m0, int& n0) {
    const int mt = gg.n_major ? lt % gg.tiles_m : lt / gg.tiles_n;
    const int nt = gg.n_major ? lt / gg.tiles_m : lt % gg.tiles_n;
    m0 = mt * TM;
    n0 = nt * TN;
}

template <int P, int TN, int KB>
__global__ void __launch_bounds__(kGThreads, 1)
    k_gemm_grouped(const GemmGroupDev* __restrict__ G, int ng, int total_tiles, int* err, unsigned long long wait_ns) {
    using CF = GCfg<P, TN, KB>;
    constexpr int S = CF::stages;
    constexpr int A_TILE = CF::A_BYTES;
    constexpr int W_TILE = CF::W_BYTES;
    extern __shared__ uint8_t smem_raw[];
    {   // an earlier launch gave up: skip (decided once per CTA, so that no thread is left at a barrier)
        __shared__ int s_abort;
        if (threadIdx.x == 0) s_abort = *(volatile int*)err;
        __syncthreads();
        if (s_abort) return;
    }
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bar0 = base + S * CF::stage_bytes;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
    auto accf_bar = [&](int a) { return bar0 + 8u * (2 * S + a); };
    auto acce_bar = [&](int a) { return bar0 + 8u * (2 * S + 2 + a); };
    const uint32_t done_bar = bar0 + 8u * (2 * S + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + S * CF::stage_bytes + 8 * (2 * S + 5));
    auto sAhi = [&](int s) { return base + s * CF::stage_bytes; };
    auto sWhi = [&](int s) { return base + s * CF::stage_bytes + A_TILE; };
    auto sAlo = [&](int s) { return base + s * CF::stage_bytes + A_TILE + W_TILE; };
    auto sWlo = [&](int s) { return base + s * CF::stage_bytes + 2 * A_TILE + W_TILE; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf_bar(a), 1);
            mbar_init(acce_bar(a), 4);     // one arrival per epilogue warp
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int kbg = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
            const int g = find_group(G, ng, t);
            const GemmGroupDev& gg = G[g];
            int m0, n0;
            tile_origin<TN>(gg, t - gg.tile_begin, m0, n0);
            const int nk = gg.K / KB;
            for (int kb = 0; kb < nk; ++kb, ++kbg) {
                const int s = kbg % S;
                if (kbg >= S) ok = mbar_wait(empty_bar(s), ((kbg / S) - 1) & 1, err, 11, true, wait_ns);
                if (!ok) break;
                mbar_expect_tx(full_bar(s), CF::stage_bytes);
                const int kc = kb * KB;
                tma_load_2d(sAhi(s), &gg.ahi, kc, m0, full_bar(s));
                tma_load_2d(sWhi(s), &gg.whi, kc, n0, full_bar(s));
                if (P == 3) {
                    tma_load_2d(sAlo(s), &gg.alo, kc, m0, full_bar(s));
                    tma_load_2d(sWlo(s), &gg.wlo, kc, n0, full_bar(s));
                }
            }
        }
        // drain: the last armed phase of every stage must land before exit
        const int armed = kbg;
        for (int k = (armed > S ? armed - S : 0); k < armed; ++k) mbar_drain(full_bar(k % S), (k / S) & 1, err, 12);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        int kbg = 0, i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x, ++i) {
            const int g = find_group(G, ng, t);
            const GemmGroupDev& gg = G[g];
            const int nk = gg.K / KB;
            int m0, n0;
            tile_origin<TN>(gg, t - gg.tile_begin, m0, n0);
            // a ragged last column tile runs MMAs only as wide as its valid columns (N % 16 == 0)
            const uint32_t idesc = idesc_n<TN>(min(TN, gg.N - n0));
            const int a = i & 1;
            if (i >= 2) ok = mbar_wait(acce_bar(a), ((i >> 1) - 1) & 1, err, 13, true, wait_ns);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(a * TN);
            for (int kb = 0; kb < nk; ++kb, ++kbg) {
                const int s = kbg % S;
                ok = mbar_wait(full_bar(s), (kbg / S) & 1, err, 14, true, wait_ns);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int k = 0; k < KB / 16; ++k) {
                    const uint32_t koff = 32u * k;    // 16 BF16 further along the swizzled row
                    const uint64_t ahi = kmajor_desc<KB>(sAhi(s) + koff), whi = kmajor_desc<KB>(sWhi(s) + koff);
                    mma_bf16_desc(acc, ahi, whi, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    if (P == 3) {
                        const uint64_t alo = kmajor_desc<KB>(sAlo(s) + koff), wlo = kmajor_desc<KB>(sWlo(s) + koff);
                        mma_bf16_desc(acc, alo, whi, idesc, 1u);
                        mma_bf16_desc(acc, ahi, wlo, idesc, 1u);
                    }
                }
                mma_commit(empty_bar(s));
            }
            if (ok) mma_commit(accf_bar(a));
        }
        mma_commit(done_bar);      // tracks every MMA issued above, also on the error path
    } else if (warp >= 2) {
        // ---------------- epilogue warps ----------------
        const int q = warp & 3;    // TMEM lane quarter this warp may access
        int i = 0;
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++i) {
            const int g = find_group(G, ng, t);
            const GemmGroupDev& gg = G[g];
            int m0, n0;
            tile_origin<TN>(gg, t - gg.tile_begin, m0, n0);
            const int a = i & 1;
            const bool have = mbar_wait(accf_bar(a), (i >> 1) & 1, err, 15, true, wait_ns);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int go = __shfl_sync(0xffffffffu, (have && *(volatile int*)err == 0) ? 1 : 0, 0);
            if (!go) break;
            const int row = m0 + q * 32 + lane;
            const uint32_t lane_addr = tmem + (uint32_t)(a * TN) + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
            for (int c = 0; c < TN && n0 + c < gg.N; c += 32) {   // columns past N were not computed
                uint32_t r[32];
                tmem_ld32(lane_addr + (uint32_t)c, r);
                const int col = n0 + c;
                if (row < gg.M && col < gg.N) {
                    float4* dst = reinterpret_cast<float4*>(gg.C + (size_t)row * gg.ldc + col);
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        if (col + 4 * v < gg.N)
                            dst[v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                                 __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(a));
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        mbar_drain(done_bar, 0, err, 16);     // every MMA has completed before TMEM is released
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TN) : "memory");
    }
}

template <int P, int TN, int KB>
int launch_grouped(cudaStream_t s, const GroupedGemm& gg, int sm_count, int* err) {
    static bool configured = false;
    if (!configured) {
        BPM_CK(cudaFuncSetAttribute(k_gemm_grouped<P, TN, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    GCfg<P, TN, KB>::smem));
        configured = true;
    }
    const int grid = std::max(1, std::min(gg.total_tiles, sm_count));
    k_gemm_grouped<P, TN, KB>
        <<<grid, kGThreads, GCfg<P, TN, KB>::smem, s>>>(gg.d_groups, gg.n_groups, gg.total_tiles, err,
                                                        gg.wait_ns ? gg.wait_ns : kWaitNs);
    BPM_CK(cudaGetLastError());
    return BPM_OK;
}

}  // namespace

int grouped_gemm_setup(GroupedGemm* gg, const std::vector<GemmOperands>& ops, int tile_n, int products, int raster,
                       int k_block, size_t l2_bytes, int pair) {
    if (pair && tile_n != 256) {
        set_error("the CTA-pair GEMM computes 256 x 256 tiles (tile_n 256)");
        return BPM_ERR_ARG;
    }
    if (k_block != 64 && k_block != 32) {
        set_error("grouped GEMM k-block must be 64 or 32");
        return BPM_ERR_ARG;
    }
    if (tile_n != 128 && tile_n != 256) {
        set_error("grouped GEMM tile width must be 128 or 256");
        return BPM_ERR_ARG;
    }
    if (raster != BPM_RASTER_AUTO && raster != BPM_RASTER_M && raster != BPM_RASTER_N) {
        set_error("unknown GEMM raster %d", raster);
        return BPM_ERR_ARG;
    }
    std::vector<GemmGroupDev> h(ops.size());
    int tiles = 0;
    for (size_t g = 0; g < ops.size(); ++g) {
        const GemmOperands& o = ops[g];
        if (o.M % tc::TM || o.K % tc::TK || o.N % 16 || o.M <= 0 || o.N <= 0) {
            set_error("grouped GEMM group %zu: M %% 128, K %% 64, N %% 16 required (M=%d N=%d K=%d)", g, o.M, o.N,
                      o.K);
            return BPM_ERR_ARG;
        }
        std::memset(&h[g], 0, sizeof(GemmGroupDev));
        // a CTA of a pair stages 128 of the tile's 256 W rows
        const int w_box = pair ? tile_n / 2 : tile_n;
        BPM_TRY(make_bf16_tensor_map(&h[g].ahi, o.Ahi, o.K, o.M, tc::TM, k_block));
        BPM_TRY(make_bf16_tensor_map(&h[g].whi, o.Whi, o.K, o.N, w_box, k_block));
        if (products == 3) {
            BPM_TRY(make_bf16_tensor_map(&h[g].alo, o.Alo, o.K, o.M, tc::TM, k_block));
            BPM_TRY(make_bf16_tensor_map(&h[g].wlo, o.Wlo, o.K, o.N, w_box, k_block));
        } else {
            h[g].alo = h[g].ahi;
            h[g].wlo = h[g].whi;
        }
        h[g].C = o.C;
        h[g].M = o.M;
        h[g].N = o.N;
        h[g].K = o.K;
        h[g].ldc = o.N;
        h[g].tiles_m = pair ? (o.M + 2 * tc::TM - 1) / (2 * tc::TM) : o.M / tc::TM;
        h[g].tiles_n = (o.N + tile_n - 1) / tile_n;
        h[g].tile_begin = tiles;
        // AUTO: N-major when the operator has more rows than the batch operand, so that the
        // larger operand is streamed once per launch and the smaller one re-read from L2
        (void)l2_bytes;
        const bool auto_n = o.N > o.M;
        h[g].n_major = raster == BPM_RASTER_N || (raster == BPM_RASTER_AUTO && auto_n) ? 1 : 0;
        tiles += h[g].tiles_m * h[g].tiles_n;
    }
    grouped_gemm_free(gg);
    BPM_CK(cudaMalloc(&gg->d_groups, h.size() * sizeof(GemmGroupDev)));
    BPM_CK(cudaMemcpy(gg->d_groups, h.data(), h.size() * sizeof(GemmGroupDev), cudaMemcpyHostToDevice));
    gg->n_groups = (int)h.size();
    gg->total_tiles = tiles;
    gg->tile_n = tile_n;
    gg->products = products;
    gg->k_block = k_block;
    gg->pair = pair;
    return BPM_OK;
}

void grouped_gemm_free(GroupedGemm* gg) {
    if (gg->d_groups) cudaFree(gg->d_groups);
    gg->d_groups = nullptr;
    gg->n_groups = gg->total_tiles = 0;
}

int grouped_gemm_launch(cudaStream_t s, GroupedGemm& gg, int sm_count, int* err) {
    if (!gg.d_groups) {
        set_error("grouped GEMM not set up");
        return BPM_ERR_STATE;
    }
    if (gg.pair) return grouped_gemm_pair_launch(s, gg, sm_count, err);
    if (gg.k_block == 32) {
        if (gg.products == 3)
            return gg.tile_n == 128 ? launch_grouped<3, 128, 32>(s, gg, sm_count, err)
                                    : launch_grouped<3, 256, 32>(s, gg, sm_count, err);
        return gg.tile_n == 128 ? launch_grouped<1, 128, 32>(s, gg, sm_count, err)
                                : launch_grouped<1, 256, 32>(s, gg, sm_count, err);
    }
    if (gg.products == 3)
        return gg.tile_n == 128 ? launch_grouped<3, 128, 64>(s, gg, sm_count, err)
                                : launch_grouped<3, 256, 64>(s, gg, sm_count, err);
    return gg.tile_n == 128 ? launch_grouped<1, 128, 64>(s, gg, sm_count, err)
                            : launch_grouped<1, 256, 64>(s, gg, sm_count, err);
}

}  // namespace bpm
