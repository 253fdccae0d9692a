// Persistent, grouped demag GEMM on CTA pairs (tcgen05 cta_group::2, sm_103a).
//
// The same product as k_gemm_grouped -- for every mesh group g of a batch,
//   C_g[M_g][N_g] = sum of the BF16 split products of A_g[M_g][K_g] and W_g[N_g][K_g]^T,
// FP32 accumulate in TMEM -- computed in 256 x 256 output tiles by the two CTAs
// of a cluster, the two SMs of one MMA: CTA r stages rows [128 r, 128 r + 128) of
// the tile's A rows and of its W rows, and the even CTA issues one MMA of
// M = 256, N = 256 that reads both CTAs' shared memory and accumulates rows
// 128 r .. 128 r + 127 of the tile in CTA r's TMEM.  Each SM thus stages and
// reads 128 W rows per k-step instead of 256, a third less shared-memory traffic
// per product than the one-SM kernel, whose tensor pipe is limited by it.
//
// Warp roles (per CTA):
//   warp 0  lane 0 streams the CTA's halves of the k-blocks with TMA into a ring
//           of shared-memory stages, each stage signalled on the CTA's own
//           barrier (so each CTA waits for its own copies alone before it gives
//           up its shared memory);
//   warp 1  allocates TMEM with the peer (two accumulators of 256 columns); in
//           the even CTA one lane issues the MMAs, tile i into accumulator i % 2,
//           and commits them to both CTAs' barriers; in the odd CTA one lane
//           forwards every landed stage to a second barrier of the stage in the
//           even CTA;
//   warps 2-5  read the CTA's accumulator rows back and store them, then arrive
//           on the even CTA's accumulator-empty barrier.
// Every wait is bounded as in k_gemm_grouped; both CTAs of a pair take the same
// abort decision before any collective step, and leave through one cluster
// barrier after every MMA (drained in both CTAs) has completed.
#include <cstring>

#include "bpm_tc_ptx.cuh"

namespace bpm {

namespace {

using namespace tc;

constexpr int kPThreads = 192;
constexpr int PTN = 256;      // output columns of a pair tile
constexpr int PHALF = 128;    // rows of A and of W staged by each CTA

template <int P, int KB>
struct PCfg {
    static constexpr int A_BYTES = PHALF * KB * 2;
    static constexpr int W_BYTES = PHALF * KB * 2;
    static constexpr int stage_bytes = (P == 3 ? 2 : 1) * (A_BYTES + W_BYTES);
    static constexpr int stages = (192 * 1024) / stage_bytes;
    static constexpr int smem = stages * stage_bytes + 1024 + 512;
    static_assert(8 * (3 * stages + 5) + 16 <= 512, "barrier area");
};

// instruction descriptor, kind::f16, BF16 x BF16 -> FP32, K-major, M = 256, N = 256
constexpr uint32_t kPairIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(PTN >> 3) << 17) |
                                ((uint32_t)(256 >> 4) << 24);

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive;\n\tbarrier.cluster.wait;" ::: "memory");
}

__device__ __forceinline__ void remote_arrive(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ int ld_cluster_s32(uint32_t cluster_addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(cluster_addr) : "memory");
    return v;
}

__device__ __forceinline__ void mma_pair(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(kPairIdesc), "r"(accumulate)
        : "memory");
}

// arrive on the barrier at this shared offset in both CTAs once the pair's MMAs issued so far complete
__device__ __forceinline__ void commit_pair(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"((uint16_t)3)
        : "memory");
}

template <int KB>
__device__ __forceinline__ uint64_t pair_desc(uint32_t addr) {
    return KB == 64 ? sw128_desc(addr) : sw64_desc(addr);
}

__device__ __forceinline__ int find_group(const GemmGroupDev* __restrict__ G, int ng, int t) {
    int g = 0;
    while (g + 1 < ng && t >= G[g + 1].tile_begin) ++g;
    return g;
}

// pair tile lt of group gg -> first row (M) and column (N); tiles_m and tiles_n count 256-tiles
__device__ __forceinline__ void pair_origin(const GemmGroupDev& gg, int lt, int& m0, int& n0) {
    const int mt = gg.n_major ? lt % gg.tiles_m : lt / gg.tiles_n;
    const int nt = gg.n_major ? lt / gg.tiles_m : lt % gg.tiles_n;
    m0 = mt * 256;
    n0 = nt * PTN;
}

template <int P, int KB>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPThreads, 1)
    k_gemm_pair(const GemmGroupDev* __restrict__ G, int ng, int total_tiles, int* err, unsigned long long wait_ns) {
    using CF = PCfg<P, KB>;
    constexpr int S = CF::stages;
    extern __shared__ uint8_t smem_raw[];
    __shared__ int s_flag;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    {   // an earlier launch gave up: both CTAs of the pair skip, decided alike from both flags
        if (threadIdx.x == 0) s_flag = *(volatile int*)err;
        cluster_sync();
        int abort = 0;
        if (threadIdx.x == 0) abort = s_flag | ld_cluster_s32(map_to(smem_u32(&s_flag), rank ^ 1u));
        abort = __syncthreads_or(abort);
        cluster_sync();        // the peer has read s_flag
        if (abort) return;
    }
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bar0 = base + S * CF::stage_bytes;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };            // this CTA's copies of stage s
    auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
    auto peer_bar = [&](int s) { return bar0 + 8u * (2 * S + s); };   // even CTA: the odd CTA's copies
    auto accf_bar = [&](int a) { return bar0 + 8u * (3 * S + a); };
    auto acce_bar = [&](int a) { return bar0 + 8u * (3 * S + 2 + a); };
    const uint32_t done_bar = bar0 + 8u * (3 * S + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + S * CF::stage_bytes + 8 * (3 * S + 5));
    auto sAhi = [&](int s) { return base + s * CF::stage_bytes; };
    auto sWhi = [&](int s) { return base + s * CF::stage_bytes + CF::A_BYTES; };
    auto sAlo = [&](int s) { return base + s * CF::stage_bytes + CF::A_BYTES + CF::W_BYTES; };
    auto sWlo = [&](int s) { return base + s * CF::stage_bytes + 2 * CF::A_BYTES + CF::W_BYTES; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
            mbar_init(peer_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf_bar(a), 1);
            mbar_init(acce_bar(a), 8);     // one arrival per epilogue warp of both CTAs (even CTA only)
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // collective with the peer CTA's warp 1
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * PTN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    cluster_sync();            // both CTAs' barriers are initialised before any remote arrival
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: this CTA's halves ----------------
        int kbg = 0;
        bool ok = true;
        for (int t = cluster; t < total_tiles && ok; t += n_clusters) {
            const int g = find_group(G, ng, t);
            const GemmGroupDev& gg = G[g];
            int m0, n0;
            pair_origin(gg, t - gg.tile_begin, m0, n0);
            const int ma = m0 + PHALF * (int)rank, nw = n0 + PHALF * (int)rank;
            const int nk = gg.K / KB;
            for (int kb = 0; kb < nk; ++kb, ++kbg) {
                const int s = kbg % S;
                if (kbg >= S) ok = mbar_wait(empty_bar(s), ((kbg / S) - 1) & 1, err, 21, true, wait_ns);
                if (!ok) break;
                mbar_expect_tx(full_bar(s), CF::stage_bytes);
                const int kc = kb * KB;
                tma_load_2d(sAhi(s), &gg.ahi, kc, ma, full_bar(s));
                tma_load_2d(sWhi(s), &gg.whi, kc, nw, full_bar(s));
                if (P == 3) {
                    tma_load_2d(sAlo(s), &gg.alo, kc, ma, full_bar(s));
                    tma_load_2d(sWlo(s), &gg.wlo, kc, nw, full_bar(s));
                }
            }
        }
        // drain: this CTA's copies land before it can give up its shared memory
        const int armed = kbg;
        for (int k = (armed > S ? armed - S : 0); k < armed; ++k) mbar_drain(full_bar(k % S), (k / S) & 1, err, 22);
    } else if (warp == 1 && lane == 0 && !leader) {
        // ---------------- forwarder (odd CTA): each landed stage to the even CTA ----------------
        // (a warp of its own: the producer's waits may suspend its warp for a while)
        int kbg = 0;
        bool ok = true;
        for (int t = cluster; t < total_tiles && ok; t += n_clusters) {
            const GemmGroupDev& gg = G[find_group(G, ng, t)];
            const int nk = gg.K / KB;
            for (int kb = 0; kb < nk; ++kb, ++kbg) {
                const int s = kbg % S;
                ok = mbar_wait(full_bar(s), (kbg / S) & 1, err, 23, true, wait_ns);
                if (!ok) break;
                remote_arrive(map_to(peer_bar(s), 0));
            }
        }
    } else if (warp == 1 && lane == 0 && leader) {
        // ---------------- MMA issuer (even CTA) ----------------
        int kbg = 0, i = 0;
        bool ok = true;
        for (int t = cluster; t < total_tiles && ok; t += n_clusters, ++i) {
            const GemmGroupDev& gg = G[find_group(G, ng, t)];
            const int nk = gg.K / KB;
            const int a = i & 1;
            if (i >= 2) ok = mbar_wait(acce_bar(a), ((i >> 1) - 1) & 1, err, 24, true, wait_ns);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(a * PTN);
            for (int kb = 0; kb < nk; ++kb, ++kbg) {
                const int s = kbg % S;
                // the odd CTA's copies of the stage have landed when its forwarder arrives (it saw
                // them complete on its own barrier first)
                ok = mbar_wait(full_bar(s), (kbg / S) & 1, err, 25, true, wait_ns) &&
                     mbar_wait(peer_bar(s), (kbg / S) & 1, err, 28, true, wait_ns);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int k = 0; k < KB / 16; ++k) {
                    const uint32_t koff = 32u * k;    // 16 BF16 further along the swizzled row
                    const uint64_t ahi = pair_desc<KB>(sAhi(s) + koff), whi = pair_desc<KB>(sWhi(s) + koff);
                    mma_pair(acc, ahi, whi, (kb > 0 || k > 0) ? 1u : 0u);
                    if (P == 3) {
                        const uint64_t alo = pair_desc<KB>(sAlo(s) + koff), wlo = pair_desc<KB>(sWlo(s) + koff);
                        mma_pair(acc, alo, whi, 1u);
                        mma_pair(acc, ahi, wlo, 1u);
                    }
                }
                commit_pair(empty_bar(s));
            }
            if (ok) commit_pair(accf_bar(a));
        }
        commit_pair(done_bar);     // tracks every MMA issued above, also on the error path
    } else if (warp >= 2) {
        // ---------------- epilogue warps: this CTA's 128 rows of each tile ----------------
        const int q = warp & 3;    // TMEM lane quarter this warp may access
        const uint32_t acce_even[2] = {map_to(acce_bar(0), 0), map_to(acce_bar(1), 0)};
        int i = 0;
        for (int t = cluster; t < total_tiles; t += n_clusters, ++i) {
            const int g = find_group(G, ng, t);
            const GemmGroupDev& gg = G[g];
            int m0, n0;
            pair_origin(gg, t - gg.tile_begin, m0, n0);
            const int a = i & 1;
            const bool have = mbar_wait(accf_bar(a), (i >> 1) & 1, err, 26, true, wait_ns);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int go = __shfl_sync(0xffffffffu, (have && *(volatile int*)err == 0) ? 1 : 0, 0);
            if (!go) break;
            const int row = m0 + PHALF * (int)rank + q * 32 + lane;
            const uint32_t lane_addr = tmem + (uint32_t)(a * PTN) + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
            for (int c = 0; c < PTN && n0 + c < gg.N; c += 32) {   // columns past N were zero operands
                uint32_t r[32];
                tmem_ld32(lane_addr + (uint32_t)c, r);
                const int col = n0 + c;
                if (row < gg.M) {
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
            if (lane == 0) remote_arrive(acce_even[a]);
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) mbar_drain(done_bar, 0, err, 27);   // every MMA into this CTA's TMEM has completed
    __syncthreads();
    cluster_sync();            // no remote arrival or shared-memory read of the pair is still to come
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * PTN) : "memory");
    }
}

template <int P, int KB>
int launch_pair(cudaStream_t s, GroupedGemm& gg, int sm_count, int* err) {
    static bool configured = false;
    if (!configured) {
        BPM_CK(cudaFuncSetAttribute(k_gemm_pair<P, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    PCfg<P, KB>::smem));
        configured = true;
    }
    if (!gg.max_pairs) {
        // pairs that can be resident at once (two SMs of one GPC each): the persistent grid
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (sm_count / 2));
        cfg.blockDim = dim3(kPThreads);
        cfg.dynamicSmemBytes = PCfg<P, KB>::smem;
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = 2;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int n = 0;
        BPM_CK(cudaOccupancyMaxActiveClusters(&n, k_gemm_pair<P, KB>, &cfg));
        if (n < 1) {
            set_error("the CTA-pair GEMM cannot be resident on this device");
            return BPM_ERR_CUDA;
        }
        gg.max_pairs = std::min(n, sm_count / 2);
    }
    const int pairs = std::max(1, std::min(gg.total_tiles, gg.max_pairs));
    k_gemm_pair<P, KB><<<2 * pairs, kPThreads, PCfg<P, KB>::smem, s>>>(gg.d_groups, gg.n_groups, gg.total_tiles,
                                                                       err, gg.wait_ns ? gg.wait_ns : kWaitNs);
    BPM_CK(cudaGetLastError());
    return BPM_OK;
}

}  // namespace

int grouped_gemm_pair_launch(cudaStream_t s, GroupedGemm& gg, int sm_count, int* err) {
    if (gg.k_block == 32)
        return gg.products == 3 ? launch_pair<3, 32>(s, gg, sm_count, err) : launch_pair<1, 32>(s, gg, sm_count, err);
    return gg.products == 3 ? launch_pair<3, 64>(s, gg, sm_count, err) : launch_pair<1, 64>(s, gg, sm_count, err);
}

}  // namespace bpm
