// Heun stage kernels of the batched LLG step, one CTA per island.
//
// LLG at 0 K (Sec. II.A; Landau-Lifshitz form with Gilbert damping):
//   dm/dt = -gamma/(1+alpha^2) [m x B + alpha m x (m x B)]
// with B = B_ex + B_an + B_d + ramp(t) (B_head + B_uniform) + B_ext, the head
// map moved at the head velocity and scaled by the field rise (Sec. II.A,
// II.C).  Heun: k1 = f(m_n, t_n), m* = N(m_n + h k1), k2 = f(m*, t_n + h),
// m_{n+1} = N(m_n + h/2 (k1 + k2)), N(v) = v/|v|.
//
// Stage 1 (predictor) and stage 2 (corrector) each stage the island's source
// state in shared memory for the exchange gather, evaluate the local field terms
// (the head map is read through L1: staging the island's map window in shared
// memory was measured slower, because the extra shared memory costs occupancy),
// take the Heun stage, renormalise, and write the demag GEMM operand of the new
// state (Ms * m, FP32 or BF16 hi/lo).  The predictor state m* is not kept in
// global memory: stage 1 writes k1 and the operand of m*, and stage 2 rebuilds
// m* = N(m_n + h k1) from m_n and k1 while staging, with the same rounding as
// stage 1 (heun_predict), so that both stages see the same m*.  Stage 2 also
// updates the volume-averaged <m_z> switch detector with a fixed-order block
// reduction.  The demag field of the stage's source state comes from the GEMM
// that ran just before the stage.  Streaming loads (state, slopes, demag field)
// are cached in L2 only, leaving L1 to the entry table and the head map.
#include <algorithm>
#include <cmath>

#include "bpm_step.cuh"

namespace bpm {

namespace {

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 v) {
    float r = rsqrtf(dot3(v, v));
    return r * v;
}

// Heun predictor N(m + h f), written out so that stage 1 and stage 2 round it alike
__device__ __forceinline__ float3 heun_predict(float3 m, float3 f, float hf) {
    const float x = __fmaf_rn(hf, f.x, m.x), y = __fmaf_rn(hf, f.y, m.y), z = __fmaf_rn(hf, f.z, m.z);
    const float r = rsqrtf(__fmaf_rn(z, z, __fmaf_rn(y, y, __fmul_rn(x, x))));
    return f3(__fmul_rn(r, x), __fmul_rn(r, y), __fmul_rn(r, z));
}

// predictor state of nodes 4q .. 4q + 3 from four-node quads of m and k1 (zero beyond n)
__device__ __forceinline__ void predict4(float4& x, float4& y, float4& z, float4 kx, float4 ky, float4 kz, float hf,
                                         int j, int n) {
    float3 v;
    v = j < n ? heun_predict(f3(x.x, y.x, z.x), f3(kx.x, ky.x, kz.x), hf) : f3(0, 0, 0);
    x.x = v.x; y.x = v.y; z.x = v.z;
    v = j + 1 < n ? heun_predict(f3(x.y, y.y, z.y), f3(kx.y, ky.y, kz.y), hf) : f3(0, 0, 0);
    x.y = v.x; y.y = v.y; z.y = v.z;
    v = j + 2 < n ? heun_predict(f3(x.z, y.z, z.z), f3(kx.z, ky.z, kz.z), hf) : f3(0, 0, 0);
    x.z = v.x; y.z = v.y; z.z = v.z;
    v = j + 3 < n ? heun_predict(f3(x.w, y.w, z.w), f3(kx.w, ky.w, kz.w), hf) : f3(0, 0, 0);
    x.w = v.x; y.w = v.y; z.w = v.z;
}

// continuous map coordinate of a point, clamped to the grid box
__device__ __forceinline__ float map_coord(float p, float origin, float h, int n) {
    float f = (p - origin) * (1.0f / h);
    return fminf(fmaxf(f, 0.f), (float)(n - 1));
}

// trilinear interpolation of the head map, clamped to the grid box; voxels come
// from the texture path with point sampling, so the arithmetic is the plain FP32
// trilinear blend of the stored values
__device__ __forceinline__ float3 trilinear(const StepArgs& a, float px, float py, float pz) {
    float fx = map_coord(px, a.mox, a.mh, a.mx), fy = map_coord(py, a.moy, a.mh, a.my),
          fz = map_coord(pz, a.moz, a.mh, a.mz);
    int ix = min((int)floorf(fx), a.mx - 2), iy = min((int)floorf(fy), a.my - 2), iz = min((int)floorf(fz), a.mz - 2);
    float wx = fx - ix, wy = fy - iy, wz = fz - iz;
    float3 acc = f3(0, 0, 0);
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                float ww = (dx ? wx : 1.f - wx) * (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
                float4 v = tex3D<float4>(a.tex, ix + dx + 0.5f, iy + dy + 0.5f, iz + dz + 0.5f);
                acc = acc + ww * f3(v.x, v.y, v.z);
            }
    return acc;
}

// effective field at node i of island b from the source state staged in smem ([3][n_pad])
__device__ __forceinline__ float3 eff_field(const StepArgs& a, int b, int i, float3 mi, const float* sm, float4 p0,
                                            float4 p1, float4 p2, float ramp, float xh, unsigned mask) {
    float3 B = f3(0, 0, 0);
    const int np = a.n_pad;
    // independent per-node loads first, so that their latency overlaps the exchange gather
    float3 hdv = f3(0, 0, 0);
    if (mask & BPM_TERM_DEMAG) {
        const float* hd = a.Hd + (size_t)b * a.kp + i;
        hdv = f3(__ldcg(hd), __ldcg(hd + np), __ldcg(hd + 2 * np));
    }
    const float4 pos = __ldg(a.node_pos + i);
    const float an0 = __ldg(&a.node_mat[i].x);
    if (mask & BPM_TERM_EXCHANGE) {
        int s = i >> 5, l = i & 31;
        int off = __ldg(a.sell_off + s);
        int nw = (__ldg(a.sell_off + s + 1) - off) >> 5;
        const int2* ep = a.sell_ent + off + l;
        float bx = 0.f, by = 0.f, bz = 0.f;
        // unrolled so that several entry loads are in flight (the loop is latency-bound)
#pragma unroll 4
        for (int e = 0; e < nw; ++e) {
            int2 c = __ldg(ep + 32 * e);
            float v = __int_as_float(c.y);
            bx += v * (sm[c.x] - mi.x);
            by += v * (sm[np + c.x] - mi.y);
            bz += v * (sm[2 * np + c.x] - mi.z);
        }
        B = B + p0.x * f3(bx, by, bz);
    }
    if (mask & BPM_TERM_ANISOTROPY) {
        float3 u = f3(p1.x, p1.y, p1.z);
        float an = an0 * p0.y;
        B = B + (an * dot3(mi, u)) * u;
    }
    if (mask & BPM_TERM_DEMAG) B = B + hdv;
    if ((mask & BPM_TERM_HEAD) && a.map) {
        B = B + ramp * trilinear(a, pos.x + p1.w - xh, pos.y + p2.x, pos.z);
    }
    if (mask & BPM_TERM_UNIFORM) {
        B = B + ramp * f3(a.uni[0], a.uni[1], a.uni[2]) + f3(p2.y, p2.z, p2.w);
    }
    return B;
}

__device__ __forceinline__ float3 llg_rhs(float3 m, float3 B, float alpha, float gp) {
    float3 mxB = cross3(m, B);
    float3 t = mxB + alpha * cross3(m, mxB);
    return (-gp) * t;
}

__device__ __forceinline__ void write_gemm_input(const StepArgs& a, int b, int i, float3 v, float msi) {
    size_t o = (size_t)b * a.kp + i;
    float x[3] = {msi * v.x, msi * v.y, msi * v.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        size_t oc = o + (size_t)c * a.n_pad;
        if (a.prec == BPM_PREC_FP32) {
            a.A32[oc] = x[c];
        } else {
            __nv_bfloat16 hi = __float2bfloat16_rn(x[c]);
            a.Ahi[oc] = hi;
            a.Alo[oc] = __float2bfloat16_rn(x[c] - __bfloat162float(hi));
        }
    }
}

// predictor state of one island from its planar m and k1 -> planar shared state
__device__ __forceinline__ void stage_predicted(const float* m, const float* k1, float* sm, int np, int n, float hf) {
    const float4* m4 = reinterpret_cast<const float4*>(m);
    const float4* k4 = reinterpret_cast<const float4*>(k1);
    float4* d4 = reinterpret_cast<float4*>(sm);
    const int nq = np / 4;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        float4 x = __ldcg(m4 + q), y = __ldcg(m4 + nq + q), z = __ldcg(m4 + 2 * nq + q);
        predict4(x, y, z, __ldcg(k4 + q), __ldcg(k4 + nq + q), __ldcg(k4 + 2 * nq + q), hf, 4 * q, n);
        d4[q] = x;
        d4[nq + q] = y;
        d4[2 * nq + q] = z;
    }
}

// planar [3][n_pad] global state -> shared memory, 16-byte copies
__device__ __forceinline__ void stage_state(const float* src, float* sm, int n_pad) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(sm);
    for (int q = threadIdx.x; q < 3 * n_pad / 4; q += blockDim.x) d4[q] = __ldcg(s4 + q);
}

__device__ __forceinline__ float block_reduce(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

__device__ __forceinline__ double step_time(const StepArgs& a, int j) {
    long long it = *a.interval;
    return a.t0 + (double)(it * a.k + j) * a.h;
}

// predictor of island b (one CTA)
__device__ __forceinline__ void stage1_body(const StepArgs& a, int b, int j) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const int np = a.n_pad;
    const size_t base = (size_t)b * 3 * np;
    const float4 p0 = a.isl[3 * b], p1 = a.isl[3 * b + 1], p2 = a.isl[3 * b + 2];
    const double t = step_time(a, j);
    const float ramp = a.rise > 0.f ? fminf(1.f, (float)(t / a.rise)) : 1.f;
    const float xh = a.x0 + a.v_nm_ps * (float)t;
    stage_state(a.m + base, sm, np);
    const float hf = (float)a.h;
    __syncthreads();
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        float3 mi = f3(sm[i], sm[np + i], sm[2 * np + i]);
        float3 B = eff_field(a, b, i, mi, sm, p0, p1, p2, ramp, xh, a.mask);
        float3 f = llg_rhs(mi, B, a.alpha, a.gp);
        float3 v = heun_predict(mi, f, hf);
        a.k1[base + i] = f.x;
        a.k1[base + np + i] = f.y;
        a.k1[base + 2 * np + i] = f.z;
        write_gemm_input(a, b, i, v, __ldg(&a.node_mat[i].y) * p0.z);
    }
}

// corrector and switch detector of island b (one CTA); red: one float per warp
__device__ __forceinline__ void stage2_body(const StepArgs& a, int b, int j, float* red) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const int np = a.n_pad;
    const size_t base = (size_t)b * 3 * np;
    const float4 p0 = a.isl[3 * b], p1 = a.isl[3 * b + 1], p2 = a.isl[3 * b + 2];
    const double t = step_time(a, j) + a.h;
    const float ramp = a.rise > 0.f ? fminf(1.f, (float)(t / a.rise)) : 1.f;
    const float xh = a.x0 + a.v_nm_ps * (float)t;
    stage_predicted(a.m + base, a.k1 + base, sm, np, a.n, (float)a.h);
    const float hh = 0.5f * (float)a.h;
    __syncthreads();
    float mzp = 0.f;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        float3 mi = f3(sm[i], sm[np + i], sm[2 * np + i]);
        const float3 mn = f3(__ldcg(a.m + base + i), __ldcg(a.m + base + np + i), __ldcg(a.m + base + 2 * np + i));
        const float3 f1 = f3(__ldcg(a.k1 + base + i), __ldcg(a.k1 + base + np + i), __ldcg(a.k1 + base + 2 * np + i));
        float3 B = eff_field(a, b, i, mi, sm, p0, p1, p2, ramp, xh, a.mask);
        float3 f2 = llg_rhs(mi, B, a.alpha, a.gp);
        float3 v = normalize3(mn + hh * (f1 + f2));
        a.m[base + i] = v.x;
        a.m[base + np + i] = v.y;
        a.m[base + 2 * np + i] = v.z;
        write_gemm_input(a, b, i, v, __ldg(&a.node_mat[i].y) * p0.z);
        mzp += __ldg(&a.node_pos[i].w) * v.z;
    }
    float mz = block_reduce(mzp, red);
    if (threadIdx.x == 0) {
        float prev = a.mz_prev[b];
        if (!a.crossed[b] && mz <= 0.f) {
            double d = (double)prev - (double)mz;
            double frac = d > 0 ? (double)prev / d : 1.0;
            a.t_sw[b] = (float)(t - a.h + a.h * frac);
            a.crossed[b] = 1;
        }
        a.mz_prev[b] = mz;
        if (!isfinite(mz)) a.status[b] |= BPM_ISLAND_NONFINITE;
    }
}

// occupancy bound: 1536 resident threads per SM (at most 40 registers each)
template <int NT>
__global__ void __launch_bounds__(NT, 1536 / NT) k_stage1(StepArgs a, int j) {
    stage1_body(a, blockIdx.x, j);
}

template <int NT>
__global__ void __launch_bounds__(NT, 1536 / NT) k_stage2(StepArgs a, int j) {
    __shared__ float red[NT / 32];
    stage2_body(a, blockIdx.x, j, red);
}

// group of CTA blockIdx.x in a launch over several mesh groups
__device__ __forceinline__ int stage_group(const StageGroups& G) {
    int g = 0;
    while (g + 1 < G.ng && (int)blockIdx.x >= G.block_begin[g + 1]) ++g;
    return g;
}

template <int NT>
__global__ void __launch_bounds__(NT, 1536 / NT) k_stage1_groups(const __grid_constant__ StageGroups G, int j) {
    const int g = stage_group(G);
    stage1_body(G.a[g], blockIdx.x - G.block_begin[g], j);
}

template <int NT>
__global__ void __launch_bounds__(NT, 1536 / NT) k_stage2_groups(const __grid_constant__ StageGroups G, int j) {
    __shared__ float red[NT / 32];
    const int g = stage_group(G);
    stage2_body(G.a[g], blockIdx.x - G.block_begin[g], j, red);
}

// ---------------------------------------------------------------------------
// Two (IPB) islands per CTA: both islands' states are staged in shared memory,
// one pass over a node's sliced-ELL entries serves both exchange sums, and the
// node data are loaded once.  The per-island arithmetic is that of eff_field,
// term by term in the same order.
// ---------------------------------------------------------------------------

// word of node j's x component of island 0 in the interleaved shared state; island q,
// component c at + 32 (3 q + c)
__device__ __forceinline__ int il_word(int j) { return (j >> 5) * (96 * kIlIslands) + (j & 31); }

// island q's planar [3][n_pad] global state -> the interleaved shared state, 16-byte copies
// (n_pad is a multiple of 32, so a copy never straddles two components)
__device__ __forceinline__ void stage_state_il(const float* src, float* sm, int np, int q) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (int k = threadIdx.x; k < 3 * np / 4; k += blockDim.x) {
        const int w = 4 * k;
        const int c = (w >= np) + (w >= 2 * np);
        const int j = w - c * np;
        *reinterpret_cast<float4*>(sm + il_word(j) + 32 * (3 * q + c)) = __ldcg(s4 + k);
    }
}

// predictor states of islands b0 .. b0 + nb - 1 -> the interleaved shared state
__device__ __forceinline__ void stage_predicted_il(const float* m, const float* k1, float* sm, int np, int n, int nb,
                                                   float hf) {
    const int nq = np / 4;
    for (int t = threadIdx.x; t < nb * nq; t += blockDim.x) {
        const int q = t / nq, qq = t - q * nq;
        const float4* m4 = reinterpret_cast<const float4*>(m + (size_t)q * 3 * np);
        const float4* k4 = reinterpret_cast<const float4*>(k1 + (size_t)q * 3 * np);
        float4 x = __ldcg(m4 + qq), y = __ldcg(m4 + nq + qq), z = __ldcg(m4 + 2 * nq + qq);
        predict4(x, y, z, __ldcg(k4 + qq), __ldcg(k4 + nq + qq), __ldcg(k4 + 2 * nq + qq), hf, 4 * qq, n);
        float* d = sm + il_word(4 * qq) + 96 * q;
        *reinterpret_cast<float4*>(d) = x;
        *reinterpret_cast<float4*>(d + 32) = y;
        *reinterpret_cast<float4*>(d + 64) = z;
    }
}

// exchange sums sum_e v_e (m_q[col_e] - m_q[i]) of node i for the IPB staged islands.  The
// entries carry the byte offset of the neighbour's word, and the components and islands sit
// at fixed distances from it, so every shared load takes an immediate offset.
template <int IPB>
__device__ __forceinline__ void exchange_sums(const StepArgs& a, int i, const float* sm, const float3 (&mi)[IPB],
                                              float3 (&bex)[IPB]) {
    static_assert(IPB == kIlIslands, "the interleaved table is laid out for kIlIslands islands");
    const int s = i >> 5, l = i & 31;
    const int off = __ldg(a.sell_off + s);
    const int nw = (__ldg(a.sell_off + s + 1) - off) >> 5;
    const int2* ep = a.sell_il + off + l;
    const char* smb = reinterpret_cast<const char*>(sm);
    float bx[IPB], by[IPB], bz[IPB];
#pragma unroll
    for (int q = 0; q < IPB; ++q) bx[q] = by[q] = bz[q] = 0.f;
#pragma unroll 4
    for (int e = 0; e < nw; ++e) {
        const int2 c = __ldg(ep + 32 * e);
        const float v = __int_as_float(c.y);
        const float* mj = reinterpret_cast<const float*>(smb + c.x);
#pragma unroll
        for (int q = 0; q < IPB; ++q) {
            bx[q] += v * (mj[32 * (3 * q)] - mi[q].x);
            by[q] += v * (mj[32 * (3 * q + 1)] - mi[q].y);
            bz[q] += v * (mj[32 * (3 * q + 2)] - mi[q].z);
        }
    }
#pragma unroll
    for (int q = 0; q < IPB; ++q) bex[q] = f3(bx[q], by[q], bz[q]);
}

// effective field of island b at node i from its exchange sum and the local terms
__device__ __forceinline__ float3 field_from_sums(const StepArgs& a, float3 mi, float3 bex, float3 hdv, float4 p0,
                                                  float4 p1, float4 p2, float4 pos, float an0, float ramp, float xh,
                                                  unsigned mask) {
    float3 B = f3(0, 0, 0);
    if (mask & BPM_TERM_EXCHANGE) B = B + p0.x * bex;
    if (mask & BPM_TERM_ANISOTROPY) {
        float3 u = f3(p1.x, p1.y, p1.z);
        float an = an0 * p0.y;
        B = B + (an * dot3(mi, u)) * u;
    }
    if (mask & BPM_TERM_DEMAG) B = B + hdv;
    if ((mask & BPM_TERM_HEAD) && a.map) {
        B = B + ramp * trilinear(a, pos.x + p1.w - xh, pos.y + p2.x, pos.z);
    }
    if (mask & BPM_TERM_UNIFORM) {
        B = B + ramp * f3(a.uni[0], a.uni[1], a.uni[2]) + f3(p2.y, p2.z, p2.w);
    }
    return B;
}

__device__ __forceinline__ float3 load_hd(const StepArgs& a, int b, int i) {
    const float* hd = a.Hd + (size_t)b * a.kp + i;
    return f3(__ldcg(hd), __ldcg(hd + a.n_pad), __ldcg(hd + 2 * a.n_pad));
}

// predictor of islands b0 .. b0 + nb - 1 (nb <= IPB); sp: [IPB][3] island parameters in smem
template <int IPB>
__device__ __forceinline__ void stage1_multi(const StepArgs& a, int b0, int j, float4* sp) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const int np = a.n_pad, S = 3 * np;
    const int nb = min(IPB, a.B - b0);
    if ((int)threadIdx.x < 3 * nb) sp[threadIdx.x] = a.isl[3 * b0 + threadIdx.x];
    const double t = step_time(a, j);
    const float ramp = a.rise > 0.f ? fminf(1.f, (float)(t / a.rise)) : 1.f;
    const float xh = a.x0 + a.v_nm_ps * (float)t;
    for (int q = 0; q < nb; ++q) stage_state_il(a.m + (size_t)(b0 + q) * S, sm, np, q);
    const float hf = (float)a.h;
    const unsigned mask = a.mask;
    __syncthreads();
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        float3 mi[IPB], bex[IPB], hdv[IPB];
        const int wi = il_word(i);
#pragma unroll
        for (int q = 0; q < IPB; ++q) {
            mi[q] = f3(sm[wi + 32 * (3 * q)], sm[wi + 32 * (3 * q + 1)], sm[wi + 32 * (3 * q + 2)]);
            hdv[q] = (mask & BPM_TERM_DEMAG) && q < nb ? load_hd(a, b0 + q, i) : f3(0, 0, 0);
        }
        const float4 pos = __ldg(a.node_pos + i);
        const float4 nm = __ldg(a.node_mat + i);
        if (mask & BPM_TERM_EXCHANGE) exchange_sums<IPB>(a, i, sm, mi, bex);
#pragma unroll
        for (int q = 0; q < IPB; ++q) {
            if (q < nb) {
            const int b = b0 + q;
            const size_t base = (size_t)b * S;
            const float4 p0 = sp[3 * q], p1 = sp[3 * q + 1], p2 = sp[3 * q + 2];
            float3 B = field_from_sums(a, mi[q], bex[q], hdv[q], p0, p1, p2, pos, nm.x, ramp, xh, mask);
            float3 f = llg_rhs(mi[q], B, a.alpha, a.gp);
            float3 v = heun_predict(mi[q], f, hf);
            a.k1[base + i] = f.x;
            a.k1[base + np + i] = f.y;
            a.k1[base + 2 * np + i] = f.z;
            write_gemm_input(a, b, i, v, nm.y * p0.z);
            }
        }
    }
}

// corrector and switch detectors of islands b0 .. b0 + nb - 1; red: [IPB][NT / 32]
template <int IPB>
__device__ __forceinline__ void stage2_multi(const StepArgs& a, int b0, int j, float4* sp, float* red) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const int np = a.n_pad, S = 3 * np;
    const int nb = min(IPB, a.B - b0);
    if ((int)threadIdx.x < 3 * nb) sp[threadIdx.x] = a.isl[3 * b0 + threadIdx.x];
    const double t = step_time(a, j) + a.h;
    const float ramp = a.rise > 0.f ? fminf(1.f, (float)(t / a.rise)) : 1.f;
    const float xh = a.x0 + a.v_nm_ps * (float)t;
    stage_predicted_il(a.m + (size_t)b0 * S, a.k1 + (size_t)b0 * S, sm, np, a.n, nb, (float)a.h);
    const float hh = 0.5f * (float)a.h;
    const unsigned mask = a.mask;
    __syncthreads();
    float mzp[IPB];
#pragma unroll
    for (int q = 0; q < IPB; ++q) mzp[q] = 0.f;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        float3 mi[IPB], bex[IPB], hdv[IPB];
        const int wi = il_word(i);
#pragma unroll
        for (int q = 0; q < IPB; ++q) {
            mi[q] = f3(sm[wi + 32 * (3 * q)], sm[wi + 32 * (3 * q + 1)], sm[wi + 32 * (3 * q + 2)]);
            hdv[q] = (mask & BPM_TERM_DEMAG) && q < nb ? load_hd(a, b0 + q, i) : f3(0, 0, 0);
        }
        const float4 pos = __ldg(a.node_pos + i);
        const float4 nm = __ldg(a.node_mat + i);
        if (mask & BPM_TERM_EXCHANGE) exchange_sums<IPB>(a, i, sm, mi, bex);
#pragma unroll
        for (int q = 0; q < IPB; ++q) {
            if (q < nb) {
            const int b = b0 + q;
            const size_t base = (size_t)b * S;
            const float4 p0 = sp[3 * q], p1 = sp[3 * q + 1], p2 = sp[3 * q + 2];
            const float3 mn = f3(__ldcg(a.m + base + i), __ldcg(a.m + base + np + i), __ldcg(a.m + base + 2 * np + i));
            const float3 f1 = f3(__ldcg(a.k1 + base + i), __ldcg(a.k1 + base + np + i), __ldcg(a.k1 + base + 2 * np + i));
            float3 B = field_from_sums(a, mi[q], bex[q], hdv[q], p0, p1, p2, pos, nm.x, ramp, xh, mask);
            float3 f2 = llg_rhs(mi[q], B, a.alpha, a.gp);
            float3 v = normalize3(mn + hh * (f1 + f2));
            a.m[base + i] = v.x;
            a.m[base + np + i] = v.y;
            a.m[base + 2 * np + i] = v.z;
            write_gemm_input(a, b, i, v, nm.y * p0.z);
            mzp[q] += pos.w * v.z;
            }
        }
    }
    // fixed-order block sums, one per island
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < IPB; ++q) {
        float v = mzp[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q * nw + (threadIdx.x >> 5)] = v;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)nb) {
        const int q = threadIdx.x, b = b0 + q;
        float mz = 0.f;
        for (int w = 0; w < nw; ++w) mz += red[q * nw + w];
        float prev = a.mz_prev[b];
        if (!a.crossed[b] && mz <= 0.f) {
            double d = (double)prev - (double)mz;
            double frac = d > 0 ? (double)prev / d : 1.0;
            a.t_sw[b] = (float)(t - a.h + a.h * frac);
            a.crossed[b] = 1;
        }
        a.mz_prev[b] = mz;
        if (!isfinite(mz)) a.status[b] |= BPM_ISLAND_NONFINITE;
    }
}

constexpr int kMultiNT = 256, kMultiIPB = 2;
// 4 CTAs (8 islands) per SM: up to 64 registers a thread; 2 x 18.8 KB of state per CTA at 1568 nodes
constexpr int kMultiMinBlocks = 4;

__global__ void __launch_bounds__(kMultiNT, kMultiMinBlocks) k_stage1m(StepArgs a, int j) {
    __shared__ float4 sp[3 * kMultiIPB];
    stage1_multi<kMultiIPB>(a, kMultiIPB * blockIdx.x, j, sp);
}
__global__ void __launch_bounds__(kMultiNT, kMultiMinBlocks) k_stage2m(StepArgs a, int j) {
    __shared__ float4 sp[3 * kMultiIPB];
    __shared__ float red[kMultiIPB * kMultiNT / 32];
    stage2_multi<kMultiIPB>(a, kMultiIPB * blockIdx.x, j, sp, red);
}
__global__ void __launch_bounds__(kMultiNT, kMultiMinBlocks) k_stage1m_groups(const __grid_constant__ StageGroups G,
                                                                             int j) {
    __shared__ float4 sp[3 * kMultiIPB];
    const int g = stage_group(G);
    stage1_multi<kMultiIPB>(G.a[g], kMultiIPB * (blockIdx.x - G.block_begin[g]), j, sp);
}
__global__ void __launch_bounds__(kMultiNT, kMultiMinBlocks) k_stage2m_groups(const __grid_constant__ StageGroups G,
                                                                             int j) {
    __shared__ float4 sp[3 * kMultiIPB];
    __shared__ float red[kMultiIPB * kMultiNT / 32];
    const int g = stage_group(G);
    stage2_multi<kMultiIPB>(G.a[g], kMultiIPB * (blockIdx.x - G.block_begin[g]), j, sp, red);
}

// ---------------------------------------------------------------------------
// Nudged elastic band (Sec. II.C, adjacent-track barrier): one CTA per image,
// image k of band d in row d * P + k.  The head field is frozen at the head
// position x0 (ramp 1).  Metric: <a, b> = sum_i w_i a_i . b_i, w_i = V_i / sum V.
// ---------------------------------------------------------------------------

constexpr unsigned kQuadTerms = BPM_TERM_EXCHANGE | BPM_TERM_ANISOTROPY | BPM_TERM_DEMAG;
constexpr unsigned kLinTerms = BPM_TERM_HEAD | BPM_TERM_UNIFORM;

// fixed-order sum of one double per thread over the CTA; every thread gets the result
template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();   // red may still be read from a previous call
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    return s;
}

// total field Bt of every image and its energy
//   E = -sum_i V_i Ms_i (B_quad,i / 2 + B_lin,i) . m_i   (J; vol_scale = sum V [nm^3] * 1e-21)
__global__ void __launch_bounds__(kStepThreads) k_neb_energy(StepArgs a, float* __restrict__ Bt,
                                                             double* __restrict__ E, double vol_scale) {
    extern __shared__ float4 smem4[];
    __shared__ double red[kStepThreads / 32];
    float* sm = reinterpret_cast<float*>(smem4);
    const int b = blockIdx.x;
    const int np = a.n_pad;
    const size_t base = (size_t)b * 3 * np;
    const float4 p0 = a.isl[3 * b], p1 = a.isl[3 * b + 1], p2 = a.isl[3 * b + 2];
    const float xh = a.x0;
    stage_state(a.m + base, sm, np);
    __syncthreads();
    double e = 0.0;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        const float3 mi = f3(sm[i], sm[np + i], sm[2 * np + i]);
        const float3 Bq = eff_field(a, b, i, mi, sm, p0, p1, p2, 1.f, xh, a.mask & kQuadTerms);
        const float3 Bl = eff_field(a, b, i, mi, sm, p0, p1, p2, 1.f, xh, a.mask & kLinTerms);
        const float3 B = Bq + Bl;
        Bt[base + i] = B.x;
        Bt[base + np + i] = B.y;
        Bt[base + 2 * np + i] = B.z;
        const float msn = __ldg(&a.node_mat[i].y) * p0.z;
        const float w = __ldg(&a.node_pos[i].w);
        e += (double)(w * msn) * (double)dot3(0.5f * Bq + Bl, mi);
    }
    const double tot = block_sum_d<kStepThreads>(e, red);
    if (threadIdx.x == 0) E[b] = -vol_scale * tot;
}

__device__ __forceinline__ float3 perp3(float3 v, float3 m) { return v + (-dot3(v, m)) * m; }
__device__ __forceinline__ float3 sub3(float3 x, float3 y) { return f3(x.x - y.x, x.y - y.y, x.z - y.z); }
__device__ __forceinline__ float3 load_state(const float* m, size_t base, int np, int i) {
    return f3(m[base + i], m[base + np + i], m[base + 2 * np + i]);
}

// one band update of every image (Jacobi: neighbours from m_in, result to m_out)
__global__ void __launch_bounds__(kStepThreads) k_neb_step(StepArgs a, NebArgs nb) {
    __shared__ double red[kStepThreads / 32];
    __shared__ int s_ci;
    const int b = blockIdx.x, P = nb.P, d = b / P, k = b - d * P;
    const int np = a.n_pad;
    const size_t S = 3 * (size_t)np, base = (size_t)b * S;
    const float msc = a.isl[3 * b].z;
    const bool end = (k == 0 || k == P - 1);
    // climbing image of this band: the interior image of highest energy
    if (threadIdx.x == 0) {
        int ci = -1;
        if (nb.climb) {
            double emax = -1e300;
            for (int q = 1; q < P - 1; ++q) {
                const double eq = nb.E[d * P + q];
                if (eq > emax) {
                    emax = eq;
                    ci = q;
                }
            }
        }
        s_ci = ci;
    }
    __syncthreads();
    const bool climbing = (k == s_ci);
    // improved tangent: weights of (m+ - m) and (m - m-) from the neighbours' energies
    float cp = 1.f, cm = 0.f;
    double inv_t = 0.0, s_ft = 0.0, spring_term = 0.0;
    if (!end) {
        const double Em = nb.E[b - 1], E0 = nb.E[b], Ep = nb.E[b + 1];
        if (Ep > E0 && E0 > Em) {
            cp = 1.f;
            cm = 0.f;
        } else if (Ep < E0 && E0 < Em) {
            cp = 0.f;
            cm = 1.f;
        } else {
            const double dmax = fmax(fabs(Ep - E0), fabs(Em - E0)), dmin = fmin(fabs(Ep - E0), fabs(Em - E0));
            cp = (float)(Ep > Em ? dmax : dmin);
            cm = (float)(Ep > Em ? dmin : dmax);
        }
        // pass 1: |t|^2, <g, t>, |m+ - m|^2, |m - m-|^2
        double stt = 0.0, sft = 0.0, dn = 0.0, dp = 0.0;
        for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
            const float w = __ldg(&a.node_pos[i].w);
            const float3 m0 = load_state(nb.m_in, base, np, i);
            const float3 mp = load_state(nb.m_in, base + S, np, i);
            const float3 mm = load_state(nb.m_in, base - S, np, i);
            const float3 dplus = sub3(mp, m0), dminus = sub3(m0, mm);
            const float3 t = perp3(cp * dplus + cm * dminus, m0);
            const float3 g = (__ldg(&a.node_mat[i].y) * msc) * perp3(load_state(nb.Bt, base, np, i), m0);
            stt += (double)(w * dot3(t, t));
            sft += (double)(w * dot3(g, t));
            dn += (double)(w * dot3(dplus, dplus));
            dp += (double)(w * dot3(dminus, dminus));
        }
        stt = block_sum_d<kStepThreads>(stt, red);
        sft = block_sum_d<kStepThreads>(sft, red);
        dn = block_sum_d<kStepThreads>(dn, red);
        dp = block_sum_d<kStepThreads>(dp, red);
        inv_t = stt > 0.0 ? 1.0 / sqrt(stt) : 0.0;
        s_ft = sft * inv_t;                                  // <g, t_hat>
        spring_term = (double)nb.spring * (sqrt(dn) - sqrt(dp));
    }
    // pass 2: band force and the normalised step
    const float c_t = climbing ? (float)(-2.0 * s_ft * inv_t) : (float)((spring_term - s_ft) * inv_t);
    float fmax_loc = 0.f;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        const float3 m0 = load_state(nb.m_in, base, np, i);
        const float msn = __ldg(&a.node_mat[i].y) * msc;
        float3 f = msn * perp3(load_state(nb.Bt, base, np, i), m0);
        if (!end) {
            const float3 mp = load_state(nb.m_in, base + S, np, i);
            const float3 mm = load_state(nb.m_in, base - S, np, i);
            const float3 t = perp3(cp * sub3(mp, m0) + cm * sub3(m0, mm), m0);
            f = f + c_t * t;
        }
        fmax_loc = fmaxf(fmax_loc, sqrtf(dot3(f, f)));
        const float3 v = normalize3(m0 + nb.step * f);
        nb.m_out[base + i] = v.x;
        nb.m_out[base + np + i] = v.y;
        nb.m_out[base + 2 * np + i] = v.z;
        write_gemm_input(a, b, i, v, msn);
    }
    for (int o = 16; o > 0; o >>= 1) fmax_loc = fmaxf(fmax_loc, __shfl_xor_sync(0xffffffffu, fmax_loc, o));
    __shared__ float redf[kStepThreads / 32];
    if ((threadIdx.x & 31) == 0) redf[threadIdx.x >> 5] = fmax_loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float f = 0.f;
        for (int w = 0; w < kStepThreads / 32; ++w) f = fmaxf(f, redf[w]);
        nb.fmax[b] = f;
    }
}

// initial band: m given (rows of [3][n_pad]) or the great circle +z -> -z through +x;
// writes the GEMM operand of every image
__global__ void __launch_bounds__(kStepThreads) k_neb_init(StepArgs a, int P, int great_circle) {
    const int b = blockIdx.x, k = b % P;
    const int np = a.n_pad;
    const size_t base = (size_t)b * 3 * np;
    const float msc = a.isl[3 * b].z;
    const float th = 3.14159265358979f * (float)k / (float)(P - 1);
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        float3 v;
        if (great_circle) {
            v = f3(sinf(th), 0.f, cosf(th));
            a.m[base + i] = v.x;
            a.m[base + np + i] = v.y;
            a.m[base + 2 * np + i] = v.z;
        } else {
            v = normalize3(load_state(a.m, base, np, i));
        }
        write_gemm_input(a, b, i, v, __ldg(&a.node_mat[i].y) * msc);
    }
}

// energy (J) and largest torque |m_i x B_i| (T) of every island at time t: the check of a
// run's state, E = -sum_i V_i Ms_i (B_quad,i / 2 + B_lin,i) . m_i with the head field moved
// and ramped to t (vol_scale = sum V [nm^3] * 1e-21), FP64 accumulation
__global__ void __launch_bounds__(kStepThreads) k_energy(StepArgs a, double t, double vol_scale,
                                                         double* __restrict__ E, float* __restrict__ torque) {
    extern __shared__ float4 smem4[];
    __shared__ double red[kStepThreads / 32];
    __shared__ float redf[kStepThreads / 32];
    float* sm = reinterpret_cast<float*>(smem4);
    const int b = blockIdx.x;
    const int np = a.n_pad;
    const float4 p0 = a.isl[3 * b], p1 = a.isl[3 * b + 1], p2 = a.isl[3 * b + 2];
    const float ramp = a.rise > 0.f ? fminf(1.f, (float)(t / a.rise)) : 1.f;
    const float xh = a.x0 + a.v_nm_ps * (float)t;
    stage_state(a.m + (size_t)b * 3 * np, sm, np);
    __syncthreads();
    double e = 0.0;
    float tq = 0.f;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        const float3 mi = f3(sm[i], sm[np + i], sm[2 * np + i]);
        const float3 Bq = eff_field(a, b, i, mi, sm, p0, p1, p2, ramp, xh, a.mask & kQuadTerms);
        const float3 Bl = eff_field(a, b, i, mi, sm, p0, p1, p2, ramp, xh, a.mask & kLinTerms);
        const float3 T = cross3(mi, Bq + Bl);
        tq = fmaxf(tq, sqrtf(dot3(T, T)));
        const float msn = __ldg(&a.node_mat[i].y) * p0.z;
        e += (double)(__ldg(&a.node_pos[i].w) * msn) * (double)dot3(0.5f * Bq + Bl, mi);
    }
    const double tot = block_sum_d<kStepThreads>(e, red);
    for (int o = 16; o > 0; o >>= 1) tq = fmaxf(tq, __shfl_xor_sync(0xffffffffu, tq, o));
    if ((threadIdx.x & 31) == 0) redf[threadIdx.x >> 5] = tq;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < kStepThreads / 32; ++w) m = fmaxf(m, redf[w]);
        E[b] = -vol_scale * tot;
        torque[b] = m;
    }
}

__global__ void __launch_bounds__(kStepThreads) k_init(StepArgs a) {
    __shared__ float red[kStepThreads / 32];
    const int b = blockIdx.x;
    const int np = a.n_pad;
    const size_t base = (size_t)b * 3 * np;
    const float4 p0 = a.isl[3 * b];
    float mzp = 0.f;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        float3 v = f3(a.m[base + i], a.m[base + np + i], a.m[base + 2 * np + i]);
        write_gemm_input(a, b, i, v, __ldg(&a.node_mat[i].y) * p0.z);
        mzp += __ldg(&a.node_pos[i].w) * v.z;
    }
    float mz = block_reduce(mzp, red);
    if (threadIdx.x == 0) {
        a.mz_prev[b] = mz;
        a.crossed[b] = mz <= 0.f ? 1 : 0;
        a.t_sw[b] = mz <= 0.f ? (float)a.t0 : -1.f;
        a.status[b] = isfinite(mz) ? 0 : BPM_ISLAND_NONFINITE;
    }
}

__global__ void __launch_bounds__(kStepThreads) k_field(StepArgs a, double t, unsigned mask, float* out) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const int b = blockIdx.x;
    const int np = a.n_pad;
    const size_t base = (size_t)b * 3 * np;
    const float4 p0 = a.isl[3 * b], p1 = a.isl[3 * b + 1], p2 = a.isl[3 * b + 2];
    const float ramp = a.rise > 0.f ? fminf(1.f, (float)(t / a.rise)) : 1.f;
    const float xh = a.x0 + a.v_nm_ps * (float)t;
    stage_state(a.m + base, sm, np);
    __syncthreads();
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        float3 mi = f3(sm[i], sm[np + i], sm[2 * np + i]);
        float3 B = eff_field(a, b, i, mi, sm, p0, p1, p2, ramp, xh, mask);
        out[base + i] = B.x;
        out[base + np + i] = B.y;
        out[base + 2 * np + i] = B.z;
    }
}

__global__ void k_tick(long long* interval) { *interval += 1; }

constexpr size_t kMaxStageSmem = 3 * sizeof(float) * kMaxNodes;

}  // namespace

size_t stage_smem_bytes(const StepArgs& a) { return 3 * sizeof(float) * (size_t)a.n_pad; }

int configure_step_kernels() {
    int smem = (int)kMaxStageSmem;
    BPM_CK(cudaFuncSetAttribute(k_stage1<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage1<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage1<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage2<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage2<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage2<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_neb_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage1_groups<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage1_groups<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage1_groups<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage2_groups<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage2_groups<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BPM_CK(cudaFuncSetAttribute(k_stage2_groups<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int smem2 = kMultiIPB * smem;
    BPM_CK(cudaFuncSetAttribute(k_stage1m, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    BPM_CK(cudaFuncSetAttribute(k_stage2m, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    BPM_CK(cudaFuncSetAttribute(k_stage1m_groups, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    BPM_CK(cudaFuncSetAttribute(k_stage2m_groups, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    return BPM_OK;
}

int stage_blocks_per_sm(int threads, int ipb, size_t smem, int* blocks) {
    int b1 = 0, b2 = 0;
    if (ipb == kMultiIPB) {
        BPM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_stage1m_groups, kMultiNT, smem));
        BPM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_stage2m_groups, kMultiNT, smem));
    } else if (threads == 128) {
        BPM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_stage1_groups<128>, 128, smem));
        BPM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_stage2_groups<128>, 128, smem));
    } else if (threads == 512) {
        BPM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_stage1_groups<512>, 512, smem));
        BPM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_stage2_groups<512>, 512, smem));
    } else {
        BPM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_stage1_groups<256>, 256, smem));
        BPM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_stage2_groups<256>, 256, smem));
    }
    *blocks = std::min(b1, b2);
    return BPM_OK;
}

int stage_islands_per_cta(const StepArgs& a) { return a.ipb == kMultiIPB ? kMultiIPB : 1; }

void launch_stage1(const StepArgs& a, int j, cudaStream_t s) {
    const size_t sm = stage_smem_bytes(a);
    if (a.ipb == kMultiIPB)
        k_stage1m<<<(a.B + kMultiIPB - 1) / kMultiIPB, kMultiNT, kMultiIPB * sm, s>>>(a, j);
    else if (a.threads == 128)
        k_stage1<128><<<a.B, 128, sm, s>>>(a, j);
    else if (a.threads == 512)
        k_stage1<512><<<a.B, 512, sm, s>>>(a, j);
    else
        k_stage1<256><<<a.B, 256, sm, s>>>(a, j);
}
void launch_stage2(const StepArgs& a, int j, cudaStream_t s) {
    const size_t sm = stage_smem_bytes(a);
    if (a.ipb == kMultiIPB)
        k_stage2m<<<(a.B + kMultiIPB - 1) / kMultiIPB, kMultiNT, kMultiIPB * sm, s>>>(a, j);
    else if (a.threads == 128)
        k_stage2<128><<<a.B, 128, sm, s>>>(a, j);
    else if (a.threads == 512)
        k_stage2<512><<<a.B, 512, sm, s>>>(a, j);
    else
        k_stage2<256><<<a.B, 256, sm, s>>>(a, j);
}
void launch_stage1_groups(const StageGroups& G, int threads, size_t smem, int j, cudaStream_t s) {
    const int blocks = G.block_begin[G.ng];
    if (G.a[0].ipb == kMultiIPB)
        k_stage1m_groups<<<blocks, kMultiNT, smem, s>>>(G, j);
    else if (threads == 128)
        k_stage1_groups<128><<<blocks, 128, smem, s>>>(G, j);
    else if (threads == 512)
        k_stage1_groups<512><<<blocks, 512, smem, s>>>(G, j);
    else
        k_stage1_groups<256><<<blocks, 256, smem, s>>>(G, j);
}
void launch_stage2_groups(const StageGroups& G, int threads, size_t smem, int j, cudaStream_t s) {
    const int blocks = G.block_begin[G.ng];
    if (G.a[0].ipb == kMultiIPB)
        k_stage2m_groups<<<blocks, kMultiNT, smem, s>>>(G, j);
    else if (threads == 128)
        k_stage2_groups<128><<<blocks, 128, smem, s>>>(G, j);
    else if (threads == 512)
        k_stage2_groups<512><<<blocks, 512, smem, s>>>(G, j);
    else
        k_stage2_groups<256><<<blocks, 256, smem, s>>>(G, j);
}
void launch_init(const StepArgs& a, cudaStream_t s) { k_init<<<a.B, kStepThreads, 0, s>>>(a); }
void launch_field(const StepArgs& a, double t, unsigned mask, float* out, cudaStream_t s) {
    k_field<<<a.B, kStepThreads, stage_smem_bytes(a), s>>>(a, t, mask, out);
}
void launch_interval_tick(long long* interval, cudaStream_t s) { k_tick<<<1, 1, 0, s>>>(interval); }

void launch_energy(const StepArgs& a, double t, double vol_scale, double* E, float* torque, cudaStream_t s) {
    k_energy<<<a.B, kStepThreads, stage_smem_bytes(a), s>>>(a, t, vol_scale, E, torque);
}
void launch_neb_init(const StepArgs& a, int P, int great_circle, cudaStream_t s) {
    k_neb_init<<<a.B, kStepThreads, 0, s>>>(a, P, great_circle);
}
void launch_neb_energy(const StepArgs& a, float* Bt, double* E, double vol_scale, cudaStream_t s) {
    k_neb_energy<<<a.B, kStepThreads, stage_smem_bytes(a), s>>>(a, Bt, E, vol_scale);
}
void launch_neb_step(const StepArgs& a, const NebArgs& nb, cudaStream_t s) {
    k_neb_step<<<a.B, kStepThreads, 0, s>>>(a, nb);
}

}  // namespace bpm
