// Head field of a saturated main pole (Sec. II.A head model; Table I geometry).
//
// Below the saturated write head the pole is uniformly magnetised at Js along
// -z, so its field is that of the magnetic surface charges on its faces:
//   mu0 H(P) = sum_k Js (m . n_k) / (4 pi)  int_k (P - Q) / |P - Q|^3 dA_Q,
// m = -z.  For a flat triangle with unit normal n (vertices counter-clockwise
// about n) the integral has the closed form
//   Omega(P) n + sum_edges m_e ln((R1 + R2 + L) / (R1 + R2 - L)),
// Omega the solid angle under which P sees the triangle (positive on the +n
// side, from the triple-product formula of the solid angle of a triangle), m_e
// the outward in-plane normal of an edge of length L, R1, R2 the distances of
// P to the edge's ends: the normal part is the solid angle, and the in-plane
// part follows from the divergence theorem in the plane, the gradient of 1/R
// over the face becoming 1/R integrated along its boundary.  The face at the
// yoke edge is the charge sheet of density Js that stands in for the yoke,
// return pole and coil.  A soft under-layer of unbounded permeability keeps the
// magnetic potential constant on its surface; the pole's mirror image in that
// plane, with charges of the opposite sign, reproduces it.
//
// A wrap-around shield of unbounded permeability (trailing and side blocks, when
// their gaps are given) keeps its surface at one magnetic potential and carries
// no net charge: its triangular
// panels get the uniform charges that satisfy this at their centroids
// (collocation), from a dense system of closed-form panel potentials factored
// by LU on the GPU in FP64.
//
// The field: one thread per voxel, FP64 over every triangle of the pole, the
// shield and their images, stored as float32 mu0 H in tesla.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "bpm_internal.cuh"

namespace bpm {

namespace {

constexpr int kMaxHeadTri = 32;      // triangles of the pole and its image
constexpr int kMaxShieldPanels = 6144;
constexpr double kPi = 3.14159265358979323846;

struct HeadTri {
    double v[3][3];  // vertices (nm), counter-clockwise about the outward normal
    double c;        // charge as mu0 sigma / (4 pi), tesla
};

struct HeadTris {
    int n;
    HeadTri t[kMaxHeadTri];
};

struct V3 {
    double x, y, z;
};
__host__ __device__ inline V3 vsub(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ inline V3 vadd(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ inline double vdot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline V3 vcross(V3 a, V3 b) {
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__host__ __device__ inline V3 vscale(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__host__ __device__ inline V3 vert(const HeadTri& t, int i) { return V3{t.v[i][0], t.v[i][1], t.v[i][2]}; }
__host__ __device__ inline V3 centroid(const HeadTri& t) {
    return vscale(1.0 / 3.0, vadd(vadd(vert(t, 0), vert(t, 1)), vert(t, 2)));
}

// int over the triangle of (P - Q) / |P - Q|^3 dA (see the file comment)
__device__ V3 tri_field(const HeadTri& tr, V3 P) {
    V3 r[3];
    double R[3];
    for (int i = 0; i < 3; ++i) {
        r[i] = vsub(vert(tr, i), P);
        R[i] = sqrt(vdot(r[i], r[i]));
    }
    const V3 nn = vcross(vsub(vert(tr, 1), vert(tr, 0)), vsub(vert(tr, 2), vert(tr, 0)));
    const V3 n = vscale(1.0 / sqrt(vdot(nn, nn)), nn);
    // signed solid angle: r_i point from P to the vertices, so the triple product is
    // negative when P lies on the +n side
    const double num = vdot(r[0], vcross(r[1], r[2]));
    const double den =
        R[0] * R[1] * R[2] + vdot(r[0], r[1]) * R[2] + vdot(r[0], r[2]) * R[1] + vdot(r[1], r[2]) * R[0];
    V3 acc = vscale(-2.0 * atan2(num, den), n);
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3;
        const V3 e = vsub(vert(tr, j), vert(tr, i));
        const double L = sqrt(vdot(e, e));
        const V3 m = vscale(1.0 / L, vcross(e, n));   // outward in the face's plane
        const double s = R[i] + R[j];
        acc = vadd(acc, vscale(log((s + L) / (s - L)), m));
    }
    return acc;
}

// int over the triangle of 1 / |P - Q| dA: with P0 the foot of P on the triangle's plane at
// signed height h, each edge (ends at s- < s+ along its unit direction t from P0's projection,
// outward in-plane normal m, distance d = (end - P0) . m to P0) adds
//   d ln((R+ + s+) / (R- + s-)) - |h| [atan(d s+ / (R0^2 + |h| R+)) - atan(d s- / (R0^2 + |h| R-))],
// R0^2 = d^2 + h^2 (the planar integral of 1/R in polar coordinates about P0, edge by edge);
// the logarithm is taken in the form (R- - s-) / (R+ - s+) where the other would cancel
__device__ double tri_potential(const HeadTri& tr, V3 P) {
    const V3 nn = vcross(vsub(vert(tr, 1), vert(tr, 0)), vsub(vert(tr, 2), vert(tr, 0)));
    const V3 n = vscale(1.0 / sqrt(vdot(nn, nn)), nn);
    const double h = vdot(vsub(P, vert(tr, 0)), n), ah = fabs(h);
    const V3 P0 = vsub(P, vscale(h, n));
    double tot = 0.0;
    for (int i = 0; i < 3; ++i) {
        const V3 a = vert(tr, i), b = vert(tr, (i + 1) % 3);
        const V3 e = vsub(b, a);
        const double L = sqrt(vdot(e, e));
        const V3 t = vscale(1.0 / L, e);
        const V3 m = vcross(t, n);
        const double sm = vdot(vsub(a, P0), t), sp = vdot(vsub(b, P0), t);
        const double d = vdot(vsub(a, P0), m);
        const V3 ra = vsub(a, P), rb = vsub(b, P);
        const double Rm = sqrt(vdot(ra, ra)), Rp = sqrt(vdot(rb, rb));
        const double R02 = d * d + h * h;
        double lg = 0.0;
        if (sp + sm >= 0.0) {
            if (Rm + sm > 0.0) lg = log((Rp + sp) / (Rm + sm));
        } else {
            lg = log((Rm - sm) / (Rp - sp));
        }
        tot += d * lg;
        if (ah > 0.0) tot -= ah * (atan2(d * sp, R02 + ah * Rp) - atan2(d * sm, R02 + ah * Rm));
    }
    return tot;
}

__global__ void k_head_field(const HeadTri* __restrict__ T, int nt, int nx, int ny, int nz, double h, double ox,
                             double oy, double oz, float* __restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)nx * ny * nz;
    if (idx >= total) return;
    const int ix = (int)(idx % nx);
    const int iy = (int)((idx / nx) % ny);
    const int iz = (int)(idx / ((long long)nx * ny));
    const V3 P{ox + h * ix, oy + h * iy, oz + h * iz};
    double bx = 0.0, by = 0.0, bz = 0.0;
    for (int k = 0; k < nt; ++k) {
        const V3 f = tri_field(T[k], P);
        bx += T[k].c * f.x;
        by += T[k].c * f.y;
        bz += T[k].c * f.z;
    }
    float* o = out + 3 * idx;
    o[0] = (float)bx;
    o[1] = (float)by;
    o[2] = (float)bz;
}

// ---- the trailing shield's boundary-element solve ----

// G[i][k] = (potential at panel i's centroid of a unit mu0 sigma on panel k, minus that of
// its image when `image`) / (4 pi)
__global__ void k_bem_matrix(const HeadTri* __restrict__ S, const HeadTri* __restrict__ Simg, int N, int image,
                             double* __restrict__ G) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * N) return;
    const int i = (int)(idx / N), k = (int)(idx % N);
    const V3 P = centroid(S[i]);
    double v = tri_potential(S[k], P);
    if (image) v -= tri_potential(Simg[k], P);
    G[idx] = v / (4.0 * kPi);
}

// b[i] = -mu0 phi of the pole's charges (and their images) at panel i's centroid
__global__ void k_pole_potential(const HeadTri* __restrict__ T, int nt, const HeadTri* __restrict__ S, int N,
                                 double* __restrict__ b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const V3 P = centroid(S[i]);
    double v = 0.0;
    for (int k = 0; k < nt; ++k) v += T[k].c * tri_potential(T[k], P);
    b[i] = -v;
}

// right-looking LU without pivoting (the self-potential dominates each row of the single-layer
// matrix): step k subtracts (G[i][k] / G[k][k]) G[k][j] from the trailing block, then scales
// column k
__global__ void k_lu_update(double* __restrict__ G, int N, int k) {
    const int j = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int i = k + 1 + blockIdx.y;
    if (j >= N || i >= N) return;
    G[(size_t)i * N + j] -= G[(size_t)i * N + k] / G[(size_t)k * N + k] * G[(size_t)k * N + j];
}
__global__ void k_lu_scale(double* __restrict__ G, int N, int k) {
    const int i = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    G[(size_t)i * N + k] /= G[(size_t)k * N + k];
}

constexpr int kSolveThreads = 1024;

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kSolveThreads / 32; ++w) s += red[w];
    return s;
}

// the two right-hand sides X[0] = b, X[1] = 1 through the unit-lower and upper factors, then
// Phi = -(A . x0) / (A . x1) (no net charge on the shield), q = x0 + Phi x1, and the panels'
// charges c = q / (4 pi) (their images -q / (4 pi)); one CTA
__global__ void __launch_bounds__(kSolveThreads) k_bem_solve(const double* __restrict__ LU, int N,
                                                            const double* __restrict__ b,
                                                            const double* __restrict__ area, double* __restrict__ X,
                                                            double* __restrict__ q, double* __restrict__ phi,
                                                            HeadTri* __restrict__ S, HeadTri* __restrict__ Simg) {
    __shared__ double red[kSolveThreads / 32];
    __shared__ double xi[2];
    double* x0 = X;
    double* x1 = X + N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        x0[i] = b[i];
        x1[i] = 1.0;
    }
    __syncthreads();
    for (int i = 0; i < N; ++i) {            // L y = rhs
        double s0 = 0.0, s1 = 0.0;
        for (int j = threadIdx.x; j < i; j += blockDim.x) {
            const double l = LU[(size_t)i * N + j];
            s0 += l * x0[j];
            s1 += l * x1[j];
        }
        s0 = block_sum(s0, red);
        s1 = block_sum(s1, red);
        if (threadIdx.x == 0) {
            x0[i] -= s0;
            x1[i] -= s1;
        }
        __syncthreads();
    }
    for (int i = N - 1; i >= 0; --i) {       // U x = y
        double s0 = 0.0, s1 = 0.0;
        for (int j = i + 1 + threadIdx.x; j < N; j += blockDim.x) {
            const double u = LU[(size_t)i * N + j];
            s0 += u * x0[j];
            s1 += u * x1[j];
        }
        s0 = block_sum(s0, red);
        s1 = block_sum(s1, red);
        if (threadIdx.x == 0) {
            const double d = LU[(size_t)i * N + i];
            x0[i] = (x0[i] - s0) / d;
            x1[i] = (x1[i] - s1) / d;
        }
        __syncthreads();
    }
    double a0 = 0.0, a1 = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        a0 += area[i] * x0[i];
        a1 += area[i] * x1[i];
    }
    a0 = block_sum(a0, red);
    a1 = block_sum(a1, red);
    if (threadIdx.x == 0) {
        xi[0] = -a0 / a1;
        *phi = xi[0];
    }
    __syncthreads();
    const double P = xi[0];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        q[i] = x0[i] + P * x1[i];
        S[i].c = q[i] / (4.0 * kPi);
        if (Simg) Simg[i].c = -q[i] / (4.0 * kPi);
    }
}

// residual of the solved system: res[0] = max_i |sum_k G0[i][k] q_k - b_i - Phi|, res[1] = max_i |b_i|
__global__ void __launch_bounds__(kSolveThreads) k_bem_residual(const double* __restrict__ G0, int N,
                                                               const double* __restrict__ b,
                                                               const double* __restrict__ q,
                                                               const double* __restrict__ phi,
                                                               double* __restrict__ res) {
    __shared__ double red[kSolveThreads / 32];
    double worst = 0.0, scale = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += G0[(size_t)i * N + k] * q[k];
        worst = fmax(worst, fabs(s - b[i] - *phi));
        scale = fmax(scale, fabs(b[i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
        scale = fmax(scale, __shfl_xor_sync(0xffffffffu, scale, o));
    }
    __shared__ double red2[kSolveThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = worst;
        red2[threadIdx.x >> 5] = scale;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double w = 0.0, sc = 0.0;
        for (int k = 0; k < kSolveThreads / 32; ++k) {
            w = fmax(w, red[k]);
            sc = fmax(sc, red2[k]);
        }
        res[0] = w;
        res[1] = sc;
    }
}

void set_tri(HeadTri& t, V3 a, V3 b, V3 c, double coef) {
    const V3 p[3] = {a, b, c};
    for (int i = 0; i < 3; ++i) {
        t.v[i][0] = p[i].x;
        t.v[i][1] = p[i].y;
        t.v[i][2] = p[i].z;
    }
    t.c = coef;
}

// Triangles of the pole (and of its image) with outward orientation and charge coefficients
int pole_triangles(const bpm_pole_geometry& g, HeadTris* T) {
    const double pi = 3.14159265358979323846, deg = pi / 180.0;
    const double w = g.pole_tip_width_nm, D = g.abs_thickness_nm, H = g.yoke_edge_nm;
    const double tt = std::tan(g.trailing_edge_angle_deg * deg), ts = std::tan(g.side_edge_angle_deg * deg);
    const double cot_taper = std::cos(g.taper_angle_deg * deg) / std::sin(g.taper_angle_deg * deg);
    const double wl = std::max(w - 2.0 * D * cot_taper, 0.1 * w);   // leading-edge width
    const double z0 = g.z_abs_nm, z1 = z0 + H;
    // ABS footprint: trailing edge at x = 0, leading edge at x = -D
    const V3 TL{0, -0.5 * w, z0}, TR{0, 0.5 * w, z0}, LR{-D, 0.5 * wl, z0}, LL{-D, -0.5 * wl, z0};
    const V3 TLu{H * tt, -(0.5 * w + H * ts), z1}, TRu{H * tt, 0.5 * w + H * ts, z1};
    const V3 LRu{-D, 0.5 * wl + H * ts, z1}, LLu{-D, -(0.5 * wl + H * ts), z1};
    // faces as corner loops: ABS, yoke edge, trailing, leading, side +y, side -y; each is split
    // along the diagonal from its first corner (the side faces from their trailing ABS corner,
    // so that the two sides mirror each other)
    const V3 quads[6][4] = {{TL, TR, LR, LL},     {TLu, TRu, LRu, LLu}, {TL, TR, TRu, TLu},
                            {LL, LR, LRu, LLu},   {TR, LR, LRu, TRu},   {TL, LL, LLu, TLu}};
    V3 C{0, 0, 0};
    const V3 all[8] = {TL, TR, LR, LL, TLu, TRu, LRu, LLu};
    for (const V3& v : all) C = V3{C.x + v.x / 8, C.y + v.y / 8, C.z + v.z / 8};
    const double js4pi = g.Js_T / (4.0 * pi);
    int n = 0;
    for (const auto& q : quads) {
        const V3 tri[2][3] = {{q[0], q[1], q[2]}, {q[0], q[2], q[3]}};
        for (const auto& t : tri) {
            V3 a = t[0], b = t[1], c = t[2];
            V3 nn = vcross(vsub(b, a), vsub(c, a));
            const double area2 = std::sqrt(vdot(nn, nn));
            if (area2 < 1e-9) continue;   // a degenerate triangle carries no charge
            const V3 mid{(a.x + b.x + c.x) / 3, (a.y + b.y + c.y) / 3, (a.z + b.z + c.z) / 3};
            if (vdot(nn, vsub(mid, C)) < 0) {
                std::swap(b, c);
                nn = vscale(-1.0, nn);
            }
            // m = -z: sigma = -(Js / mu0) n_z
            set_tri(T->t[n++], a, b, c, -js4pi * nn.z / area2);
        }
    }
    if (g.sul_image) {
        const int np = n;
        for (int k = 0; k < np; ++k) {
            const HeadTri& s = T->t[k];
            V3 p[3];
            for (int i = 0; i < 3; ++i) p[i] = V3{s.v[i][0], s.v[i][1], 2.0 * g.z_sul_nm - s.v[i][2]};
            // the mirror reverses the winding: swap two vertices so that the image's normal is the
            // mirrored outward normal; the image charge has the opposite sign
            set_tri(T->t[n++], p[0], p[2], p[1], -s.c);
        }
    }
    T->n = n;
    return BPM_OK;
}

// Panels of the shield: the trailing block stands on the ABS with its leading face parallel to
// the pole's trailing face at the gap, shield_thickness high, kShieldDepth deep down-track and
// kShieldMargin wider than the pole tip on each side (a parallelepiped sheared along x by the
// trailing edge angle); each side block (with a side shield gap) has its inner face parallel to
// the pole's flared side at that gap, runs down-track from kSideLead behind the leading edge to
// kSideClear short of the trailing block, and reaches out to the trailing block's cross-track
// extent (a parallelepiped sheared along y by the side edge angle).  The blocks form one body.
// Each face is a grid of about panel x panel parallelograms, each split along its diagonal from
// its first corner into two triangles, wound outward.  area: the triangles' areas (nm^2).
constexpr double kShieldDepth = 30.0, kShieldMargin = 40.0, kSideLead = 10.0, kSideClear = 0.5;

struct Block {
    V3 O, ex, ey, ez;
};

void shield_panels(const bpm_pole_geometry& g, double panel, std::vector<HeadTri>& P, std::vector<double>& area) {
    const double deg = kPi / 180.0;
    const double tt = std::tan(g.trailing_edge_angle_deg * deg), ts = std::tan(g.side_edge_angle_deg * deg);
    const double w = g.pole_tip_width_nm, W = w + 2.0 * kShieldMargin, T = g.shield_thickness_nm;
    std::vector<Block> blocks;
    if (g.trailing_shield_gap_nm > 0.f)
        blocks.push_back(Block{V3{g.trailing_shield_gap_nm, -0.5 * W, g.z_abs_nm}, V3{kShieldDepth, 0, 0},
                               V3{0, W, 0}, V3{T * tt, 0, T}});
    if (g.side_shield_gap_nm > 0.f) {
        const double x0 = -g.abs_thickness_nm - kSideLead;
        const double x1 = std::max(0.0, (double)g.trailing_shield_gap_nm) - kSideClear;
        const double inner = 0.5 * w + g.side_shield_gap_nm, reach = 0.5 * W - inner;
        blocks.push_back(Block{V3{x0, inner, g.z_abs_nm}, V3{x1 - x0, 0, 0}, V3{0, reach, 0}, V3{0, T * ts, T}});
        blocks.push_back(Block{V3{x0, -0.5 * W, g.z_abs_nm}, V3{x1 - x0, 0, 0}, V3{0, reach, 0},
                               V3{0, -T * ts, T}});
    }
    P.clear();
    area.clear();
    for (const Block& bk : blocks) {
        const V3 O = bk.O, ex = bk.ex, ey = bk.ey, ez = bk.ez;
        const V3 C = vadd(O, vscale(0.5, vadd(vadd(ex, ey), ez)));
        const V3 faces[6][3] = {{O, ex, ey},          {vadd(O, ez), ex, ey}, {O, ey, ez},
                                {vadd(O, ex), ey, ez}, {O, ex, ez},          {vadd(O, ey), ex, ez}};
        for (const auto& f : faces) {
            const V3 F0 = f[0], U = f[1], V = f[2];
            const int nu = std::max(1, (int)std::ceil(std::sqrt(vdot(U, U)) / panel - 1e-9));
            const int nv = std::max(1, (int)std::ceil(std::sqrt(vdot(V, V)) / panel - 1e-9));
            for (int i = 0; i < nu; ++i)
                for (int j = 0; j < nv; ++j) {
                    auto pt = [&](int a, int b) {
                        return vadd(F0, vadd(vscale((double)a / nu, U), vscale((double)b / nv, V)));
                    };
                    const V3 p00 = pt(i, j), p10 = pt(i + 1, j), p11 = pt(i + 1, j + 1), p01 = pt(i, j + 1);
                    const V3 tri[2][3] = {{p00, p10, p11}, {p00, p11, p01}};
                    for (const auto& t : tri) {
                        V3 a = t[0], b = t[1], c = t[2];
                        V3 nn = vcross(vsub(b, a), vsub(c, a));
                        const V3 mid = vscale(1.0 / 3.0, vadd(vadd(a, b), c));
                        if (vdot(nn, vsub(mid, C)) < 0) std::swap(b, c);
                        HeadTri h{};
                        set_tri(h, a, b, c, 0.0);
                        P.push_back(h);
                        area.push_back(0.5 * std::sqrt(vdot(nn, nn)));
                    }
                }
        }
    }
}

// the mirror image of a triangle in z = z_sul (winding kept outward), charge `coef`
HeadTri mirrored(const HeadTri& s, double z_sul, double coef) {
    V3 p[3];
    for (int i = 0; i < 3; ++i) p[i] = V3{s.v[i][0], s.v[i][1], 2.0 * z_sul - s.v[i][2]};
    HeadTri t{};
    set_tri(t, p[0], p[2], p[1], coef);
    return t;
}

// device buffers of one solve, freed on every exit
struct HeadBufs {
    cudaStream_t s = nullptr;
    HeadTri* T = nullptr;
    double *G = nullptr, *G0 = nullptr, *b = nullptr, *area = nullptr, *X = nullptr, *q = nullptr, *res = nullptr;
    float* out = nullptr;
    ~HeadBufs() {
        void* ptrs[] = {T, G, G0, b, area, X, q, res, out};
        for (void* p : ptrs)
            if (p) cudaFreeAsync(p, s);
    }
};

template <class X>
int head_alloc(HeadBufs& hb, X** p, size_t count) {
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(1, count) * sizeof(X), hb.s);
    if (e != cudaSuccess) {
        set_error("head-field buffers: %s", cudaGetErrorString(e));
        return BPM_ERR_OOM;
    }
    return BPM_OK;
}

}  // namespace

}  // namespace bpm

using namespace bpm;

extern "C" int bpm_head_field_solve(bpm_ctx* ctx, const bpm_pole_geometry* g, int32_t nx, int32_t ny, int32_t nz,
                                    float h_nm, const float origin_nm[3], float* B_T, int on_device) {
    if (!ctx || !g || !origin_nm || !B_T || nx < 1 || ny < 1 || nz < 1 || !(h_nm > 0.f) ||
        (long long)nx * ny * nz > (1LL << 28)) {
        set_error("bad head-field arguments (context, geometry, grid of 1 .. 2^28 voxels, h > 0, output)");
        return BPM_ERR_ARG;
    }
    const bpm_pole_geometry& G = *g;
    const bool geo_ok = G.pole_tip_width_nm > 0.f && G.abs_thickness_nm > 0.f && G.yoke_edge_nm > 0.f &&
                        G.Js_T > 0.f && G.trailing_edge_angle_deg >= 0.f && G.trailing_edge_angle_deg < 80.f &&
                        G.side_edge_angle_deg >= 0.f && G.side_edge_angle_deg < 80.f && G.taper_angle_deg > 0.f &&
                        G.taper_angle_deg <= 90.f && (!G.sul_image || G.z_sul_nm < G.z_abs_nm);
    if (!geo_ok) {
        set_error("bad pole geometry (positive sizes and Js, edge angles in [0, 80) deg, taper in (0, 90] deg, "
                  "under-layer below the ABS)");
        return BPM_ERR_ARG;
    }
    const double z_top = (double)origin_nm[2] + (double)h_nm * (nz - 1);
    if (!(z_top < G.z_abs_nm) || (G.sul_image && !((double)origin_nm[2] > G.z_sul_nm))) {
        set_error("the head-field grid must lie below the ABS (and above the under-layer)");
        return BPM_ERR_ARG;
    }
    const bool shield = G.trailing_shield_gap_nm > 0.f || G.side_shield_gap_nm > 0.f;
    const double panel = G.shield_panel_nm > 0.f ? G.shield_panel_nm : 2.0;
    if (shield && (!(G.shield_thickness_nm > 0.f) || panel < 0.5 || !(G.side_shield_gap_nm < kShieldMargin))) {
        set_error("a shield needs a positive thickness, panels of at least 0.5 nm and a side gap below %g nm",
                  kShieldMargin);
        return BPM_ERR_ARG;
    }
    HeadTris pole{};
    BPM_TRY(pole_triangles(G, &pole));
    std::vector<HeadTri> S;
    std::vector<double> area;
    if (shield) {
        shield_panels(G, panel, S, area);
        if ((int)S.size() > kMaxShieldPanels) {
            set_error("%zu shield panels, more than %d: use larger panels", S.size(), kMaxShieldPanels);
            return BPM_ERR_ARG;
        }
    }
    const int N = (int)S.size(), img = G.sul_image ? 1 : 0;
    // all triangles: the pole (and its image), then the shield panels, then their images
    std::vector<HeadTri> all(pole.t, pole.t + pole.n);
    all.insert(all.end(), S.begin(), S.end());
    if (img)
        for (const HeadTri& p : S) all.push_back(mirrored(p, G.z_sul_nm, 0.0));
    BPM_CK(cudaSetDevice(ctx->device));
    HeadBufs hb;
    hb.s = ctx->stream;
    cudaStream_t st = ctx->stream;
    BPM_TRY(head_alloc(hb, &hb.T, all.size()));
    BPM_CK(cudaMemcpyAsync(hb.T, all.data(), all.size() * sizeof(HeadTri), cudaMemcpyHostToDevice, st));
    if (N > 0) {
        HeadTri* dS = hb.T + pole.n;
        HeadTri* dSimg = img ? dS + N : nullptr;
        const size_t NN = (size_t)N * N;
        BPM_TRY(head_alloc(hb, &hb.G, NN));
        BPM_TRY(head_alloc(hb, &hb.G0, NN));
        BPM_TRY(head_alloc(hb, &hb.b, N));
        BPM_TRY(head_alloc(hb, &hb.area, N));
        BPM_TRY(head_alloc(hb, &hb.X, 2 * (size_t)N));
        BPM_TRY(head_alloc(hb, &hb.q, N));
        BPM_TRY(head_alloc(hb, &hb.res, 3));
        BPM_CK(cudaMemcpyAsync(hb.area, area.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
        k_bem_matrix<<<(unsigned)((NN + 255) / 256), 256, 0, st>>>(dS, dSimg, N, img, hb.G);
        k_pole_potential<<<(N + 127) / 128, 128, 0, st>>>(hb.T, pole.n, dS, N, hb.b);
        BPM_CK(cudaMemcpyAsync(hb.G0, hb.G, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k + 1 < N; ++k) {
            const int rest = N - k - 1;
            k_lu_update<<<dim3((rest + 255) / 256, rest), 256, 0, st>>>(hb.G, N, k);
            k_lu_scale<<<(rest + 255) / 256, 256, 0, st>>>(hb.G, N, k);
        }
        k_bem_solve<<<1, kSolveThreads, 0, st>>>(hb.G, N, hb.b, hb.area, hb.X, hb.q, hb.res + 2, dS, dSimg);
        k_bem_residual<<<1, kSolveThreads, 0, st>>>(hb.G0, N, hb.b, hb.q, hb.res + 2, hb.res);
        BPM_CK(cudaGetLastError());
        double res[2] = {0, 0};
        BPM_CK(cudaMemcpyAsync(res, hb.res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        BPM_CK(cudaStreamSynchronize(st));
        if (!(res[0] <= 1e-8 * res[1])) {
            set_error("shield solve residual %.3g of %.3g", res[0], res[1]);
            return BPM_ERR_UNSTABLE;
        }
    }
    const size_t count = (size_t)nx * ny * nz;
    float* dst = B_T;
    if (!on_device) {
        BPM_TRY(head_alloc(hb, &hb.out, count * 3));
        dst = hb.out;
    }
    const int threads = 256;
    k_head_field<<<(unsigned)((count + threads - 1) / threads), threads, 0, st>>>(
        hb.T, (int)all.size(), nx, ny, nz, h_nm, origin_nm[0], origin_nm[1], origin_nm[2], dst);
    BPM_CK(cudaGetLastError());
    if (!on_device) {
        BPM_CK(cudaMemcpyAsync(B_T, dst, count * 3 * sizeof(float), cudaMemcpyDeviceToHost, st));
        BPM_CK(cudaStreamSynchronize(st));
    }
    return BPM_OK;
}
