// Internal declarations shared by the translation units of libbpmllg.so.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/bpm.h"

namespace bpm {

constexpr double kMu0 = 1.25663706143591729e-6;       // 4 pi 1e-7 T m / A
constexpr double kGammaPs = 1.76085963023e-1;         // rad / (ps T)
constexpr int kMaxNodes = 8192;
constexpr int kNodePad = 32;                           // n_pad multiple: whole 32-row exchange slices
constexpr int kKPad = 64;                              // demag GEMM K multiple (one 128-byte BF16 k-block)
constexpr int kIslandPad = 128;                        // batch rows padded to the GEMM M tile

void set_error(const char* fmt, ...);

#define BPM_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            bpm::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                  \
                           cudaGetErrorString(e_));                                    \
            return (e_ == cudaErrorMemoryAllocation) ? BPM_ERR_OOM : BPM_ERR_CUDA;     \
        }                                                                              \
    } while (0)

#define BPM_TRY(expr)              \
    do {                           \
        int r_ = (expr);           \
        if (r_ != BPM_OK) return r_; \
    } while (0)

// Islands per CTA of the interleaved stage kernels.  Their shared state holds
// component c of node j of island q at word ((j >> 5) * 3 * kIlIslands + 3 q + c) * 32 + (j & 31),
// so that the three components of both islands sit at fixed distances from node j's word.
constexpr int kIlIslands = 2;

// Chains of islands a batch's interval graph may run on separate streams (tuning streams).
constexpr int kMaxChains = 4;

// Position (nm) and lumped volume weight V_i / sum V of one node, FP64.
struct NodeF64 {
    double x, y, z, w;
};

// Device-resident operators of one island mesh.
struct Mesh {
    int n = 0, n_pad = 0, n_tets = 0, nb = 0, nnz = 0;
    // demag GEMM width: the operand row of an island holds its three component planes
    // [c n_pad, c n_pad + n) and zeros up to k_pad = 3 n_pad rounded up to kKPad
    int k_pad = 0;
    // per node (padded to n_pad; padding nodes have w = 0 and no neighbours)
    float4* node_pos = nullptr;   // x, y, z (nm), w_i = V_i / sum V
    float4* node_mat = nullptr;   // 2 Ku_i / Ms_i (T), Ms_i (MA/m), 0, 0
    // exchange operator, difference form, sliced ELL with 32-row slices:
    // B_ex,i = (1/Ms_scale) sum_e val_e (m_{col_e} - m_i); padding entries val = 0, col = i
    int n_slices = 0;
    int* sell_off = nullptr;      // [n_slices + 1] first entry of each slice
    int2* sell_ent = nullptr;     // (col, float bits of val), entry e of row 32 s + l at off[s] + 32 e + l
    // the same entries with col replaced by the byte offset of node col's x component in the
    // interleaved shared state of the two-island stage kernels (see kIlIslands)
    int2* sell_il = nullptr;
    // demag operator -mu0*1e6*N, row c*n_pad+i, column c'*n_pad+k (T per MA/m); rows and
    // columns from 3 n_pad to k_pad are zero
    float* N32 = nullptr;         // [K][K], K = k_pad
    __nv_bfloat16* Nhi = nullptr; // [K][K]
    __nv_bfloat16* Nlo = nullptr; // [K][K]
    double* N64 = nullptr;        // [3n][3n] compact, H = -N M (only with BPM_MESH_KEEP_F64)
    // FP64 copies for the plain FP64 form: exchange CSR in difference form, c_ij (T per unit m,
    // c_ii = 0), and per node (x, y, z, V_i / sum V) and (2 Ku_i / Ms_i in T, Ms_i in A/m)
    int* csr_rowptr = nullptr;    // [n + 1]
    int* csr_col = nullptr;       // [nnz]
    double* csr_c64 = nullptr;    // [nnz]
    NodeF64* node64 = nullptr;    // [n]
    double2* mat64 = nullptr;     // [n]
    // host copies for export
    std::vector<int> rowptr, col; // CSR pattern incl. diagonal
    std::vector<float> exch_val;  // c_ij per CSR entry (0 on the diagonal)
    std::vector<double> V, Ms, Ku;
    double an_max = 0;            // max_i 2 Ku_i / Ms_i (T)
    double ms_max = 0;            // max_i Ms_i (A/m)
    bpm_mesh_info info{};
    int K() const { return k_pad; }
};

struct HeadMap {
    float4* B = nullptr;          // [nz][ny][nx] (Bx, By, Bz, 0)
    cudaArray_t arr = nullptr;    // the same voxels in a 3-D array, read through the texture path
    cudaTextureObject_t tex = 0;  // point sampling, unnormalised coordinates, clamped
    int nx = 0, ny = 0, nz = 0;
    float h = 1.f;
    float origin[3] = {0, 0, 0};
    double max_norm = 0;          // largest |B| of a voxel (T)
};

struct Mlp;
void free_mlp(Mlp* m);
struct Gp;
void free_gp(Gp* g);

}  // namespace bpm

struct bpm_ctx {
    int device = 0;
    int sm_count = 0;
    size_t l2_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<bpm::Mesh*> meshes;
    std::vector<bpm::HeadMap*> maps;
    std::vector<bpm::Mlp*> mlps;
    std::vector<bpm::Gp*> gps;
};

namespace bpm {

// Integrator step count of a run (bpm_stable_substeps): *k (>= 1) and the field bound (T)
int stable_substeps(bpm_ctx* ctx, const bpm_island* isl, int B, const bpm_run_params* p, int* k, double* bound);
// Heun steps of a run: p->substeps, or the stable count when p->substeps is 0
int run_substeps(bpm_ctx* ctx, const bpm_island* isl, int B, const bpm_run_params* p, int* k);

// assembly (bpm_assemble.cu)
int assemble_mesh(bpm_ctx* ctx, Mesh* M, const double* xyz, const int32_t* tets, int32_t n_tets,
                  const int32_t* region, const bpm_region_mat* mats, int32_t n_regions,
                  uint32_t flags);
void free_mesh(Mesh* M);

// epilogues of the tensor-core GEMM (C = A W^T, BF16 operands, FP32 accumulate)
enum { TC_EPI_STORE = 0, TC_EPI_BIAS_GELU = 1, TC_EPI_BIAS_OUT = 2, TC_EPI_GELU_BWD = 3 };
struct TcEpilogue {
    float* C = nullptr;            // FP32 [row][col] (STORE: result; BIAS_GELU: pre-activation z; BIAS_OUT: logits/probs)
    int ldc = 0;
    const float* bias = nullptr;   // [cols_valid]
    __nv_bfloat16* H = nullptr;    // BF16 [row][col] (BIAS_GELU: activation; GELU_BWD: dz)
    int ldh = 0;
    __nv_bfloat16* HT = nullptr;   // BF16 [col][row], the transposed copy (optional)
    int ldht = 0;
    const float* Zin = nullptr;    // GELU_BWD: pre-activation [row][col]
    int ldz = 0;
    float* colsum = nullptr;       // GELU_BWD: per (32-row block, column) partial sums
    int ldcs = 0;
    int rows_valid = 0, cols_valid = 0;
    int sigmoid = 0;               // BIAS_OUT: apply the logistic function
};
int gemm_tc(cudaStream_t s, int epi, int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* W,
            const TcEpilogue& e, int* err_flag);

// grouped persistent tensor-core GEMM (bpm_gemm_grouped.cu): one launch over the
// output tiles of every mesh group of a batch
struct GemmGroupDev {   // CUtensorMap members carry the 64-byte alignment TMA needs
    CUtensorMap ahi, alo, whi, wlo;   // 128 B each, 64-byte aligned
    float* C;
    int M, N, K, ldc;
    int tiles_m, tiles_n;             // output tiles of this group along M and N
    int tile_begin;                   // first tile of this group in the launch's list
    int n_major;                      // tile order: 1 = consecutive tiles share the W rows
};
struct GemmOperands {
    const __nv_bfloat16 *Ahi, *Alo, *Whi, *Wlo;
    float* C;
    int M, N, K;
};
struct GroupedGemm {
    GemmGroupDev* d_groups = nullptr;
    int n_groups = 0, total_tiles = 0, tile_n = 256, products = 3, k_block = 64;
    unsigned long long wait_ns = 0;   // limit of the non-drain waits (0: the default)
    int pair = 0;                     // 1: 256 x 256 tiles on CTA pairs (tcgen05 cta_group::2)
    int max_pairs = 0;                // co-resident CTA pairs of the pair kernel (0: not yet queried)
};
// k_block: K depth of one pipeline stage, 64 (128-byte swizzle) or 32 (64-byte swizzle, twice the stages)
// pair: 256 x 256 output tiles computed by the two CTAs of a cluster (bpm_gemm_pair.cu)
int grouped_gemm_setup(GroupedGemm* gg, const std::vector<GemmOperands>& ops, int tile_n, int products, int raster,
                       int k_block, size_t l2_bytes, int pair = 0);
int grouped_gemm_pair_launch(cudaStream_t s, GroupedGemm& gg, int sm_count, int* err);
void grouped_gemm_free(GroupedGemm* gg);
int grouped_gemm_launch(cudaStream_t s, GroupedGemm& gg, int sm_count, int* err);
// TMA map of a row-major BF16 [rows][inner] matrix, boxes of box_rows x box_inner (64 or 32)
int make_bf16_tensor_map(CUtensorMap* map, const void* ptr, int inner, int rows, int box_rows, int box_inner = 64);

// demag GEMMs: C[M_rows][Nout] = A[M_rows][K] * W[Nout][K]^T, row strides lda/ldw/ldc (elements)
int gemm_f32_nt(cudaStream_t s, int M_rows, int Nout, int K, const float* A, int lda,
                const float* W, int ldw, float* C, int ldc);
int gemm_bf16x3_simt(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* Ahi,
                     const __nv_bfloat16* Alo, const __nv_bfloat16* Whi, const __nv_bfloat16* Wlo,
                     float* C, int products);

}  // namespace bpm
