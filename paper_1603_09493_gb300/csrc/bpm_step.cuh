// Per-island Heun stage kernels: declarations shared by the API layer.
#pragma once
#include "bpm_internal.cuh"

namespace bpm {

struct StepArgs {
    int B, n, n_pad;
    int kp;                   // row stride of Hd and the GEMM operand (k_pad >= 3 n_pad)
    const float4* node_pos;   // [n_pad] x, y, z, w
    const float4* node_mat;   // [n_pad] 2Ku/Ms (T), Ms (MA/m)
    const int* sell_off;
    const int2* sell_ent;
    const int2* sell_il;      // sell_ent with shared-state byte offsets (two-island kernels)
    const float4* isl;        // [B][3] (1/Ms_s, Ku_s/Ms_s, Ms_s, 0), (u, pos_x), (pos_y, Hext)
    const float4* map;        // head map (linear copy) or nullptr: no head field
    cudaTextureObject_t tex;  // head map voxels for the lookups
    int mx, my, mz;
    float mh, mox, moy, moz;
    float* m;                 // [Bp][3][n_pad]
    float* k1;                // predictor slope
    const float* Hd;          // demag field of the GEMM input state, tesla, [Bp][kp]
    float* A32;               // GEMM input (FP32), [Bp][kp], Ms * m in MA/m (planes at c n_pad)
    __nv_bfloat16* Ahi;       // GEMM input BF16 hi/lo split
    __nv_bfloat16* Alo;
    int prec;
    float* mz_prev;           // [B] detector state
    float* t_sw;
    int* crossed;
    int* status;
    const long long* interval;  // device interval counter
    double t0, h;
    int k;                    // steps per interval
    float alpha, gp;          // damping, gamma/(1+alpha^2) in rad/(ps T)
    float rise, v_nm_ps, x0;
    float uni[3];
    unsigned mask;
    int threads;              // CTA size of the stage kernels: 128, 256 or 512 (autotuned)
    int ipb;                  // islands per stage CTA: 1, or 2 (256 threads; autotuned)
};

constexpr int kStepThreads = 256;

// one stage launch over several mesh groups of a batch: CTAs
// [block_begin[g], block_begin[g + 1]) integrate the islands of group g (one or
// two islands per CTA, as a.ipb of the groups says; all groups of a launch agree).  Passed
// by value (a grid-constant kernel parameter, under 10 KB); the groups of one
// launch share the CTA size, and the dynamic shared memory is the largest
// group's.
constexpr int kMaxStageGroups = 32;
struct StageGroups {
    int ng;
    int block_begin[kMaxStageGroups + 1];
    StepArgs a[kMaxStageGroups];
};

void launch_stage1(const StepArgs& a, int j, cudaStream_t s);
void launch_stage2(const StepArgs& a, int j, cudaStream_t s);
void launch_stage1_groups(const StageGroups& G, int threads, size_t smem, int j, cudaStream_t s);
void launch_stage2_groups(const StageGroups& G, int threads, size_t smem, int j, cudaStream_t s);
size_t stage_smem_bytes(const StepArgs& a);
// resident CTAs per SM of the grouped stage kernels at this CTA size, islands per CTA and
// shared memory
int stage_blocks_per_sm(int threads, int ipb, size_t smem, int* blocks);
// islands per stage CTA of these arguments (1 or 2)
int stage_islands_per_cta(const StepArgs& a);
void launch_init(const StepArgs& a, cudaStream_t s);
void launch_field(const StepArgs& a, double t, unsigned mask, float* out, cudaStream_t s);
void launch_interval_tick(long long* interval, cudaStream_t s);

// nudged elastic band (rows of a.m are images; a.x0 is the frozen head position)
struct NebArgs {
    int P;                    // images per band (rows d * P .. d * P + P - 1)
    int climb;                // 1: the highest interior image of each band climbs
    float step;               // m <- N(m + step * force), force in MA/m x T
    float spring;             // spring constant, MA/m x T per unit of weighted distance
    const double* E;          // [rows] energies of m_in (J)
    const float* Bt;          // [rows][3][n_pad] effective field of m_in (T)
    const float* m_in;        // [rows][3][n_pad]
    float* m_out;             // [rows][3][n_pad]
    float* fmax;              // [rows] max_i |band force_i| of this update
};
// energy (J) and largest torque |m x B| (T) of each island at time t (a.mask selects the terms)
void launch_energy(const StepArgs& a, double t, double vol_scale, double* E, float* torque, cudaStream_t s);
void launch_neb_init(const StepArgs& a, int P, int great_circle, cudaStream_t s);
void launch_neb_energy(const StepArgs& a, float* Bt, double* E, double vol_scale, cudaStream_t s);
void launch_neb_step(const StepArgs& a, const NebArgs& nb, cudaStream_t s);
int configure_step_kernels();

}  // namespace bpm
