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
// One thread per voxel, FP64 over every triangle of the pole and its image (at
// most 24), the result stored as float32 mu0 H in tesla.
#include <algorithm>
#include <cmath>
#include <utility>

#include "bpm_internal.cuh"

namespace bpm {

namespace {

constexpr int kMaxHeadTri = 32;

struct HeadTri {
    double v[3][3];  // vertices (nm), counter-clockwise about the outward normal
    double c;        // Js (m . n) / (4 pi), tesla
};

struct HeadTris {
    int n;
    HeadTri t[kMaxHeadTri];
};

struct V3 {
    double x, y, z;
};
__host__ __device__ inline V3 vsub(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ inline double vdot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline V3 vcross(V3 a, V3 b) {
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__host__ __device__ inline V3 vscale(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__host__ __device__ inline V3 vert(const HeadTri& t, int i) { return V3{t.v[i][0], t.v[i][1], t.v[i][2]}; }

__global__ void k_head_field(const __grid_constant__ HeadTris T, int nx, int ny, int nz, double h, double ox,
                             double oy, double oz, float* __restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)nx * ny * nz;
    if (idx >= total) return;
    const int ix = (int)(idx % nx);
    const int iy = (int)((idx / nx) % ny);
    const int iz = (int)(idx / ((long long)nx * ny));
    const V3 P{ox + h * ix, oy + h * iy, oz + h * iz};
    double bx = 0.0, by = 0.0, bz = 0.0;
    for (int k = 0; k < T.n; ++k) {
        const HeadTri& tr = T.t[k];
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
        const double den = R[0] * R[1] * R[2] + vdot(r[0], r[1]) * R[2] + vdot(r[0], r[2]) * R[1] +
                           vdot(r[1], r[2]) * R[0];
        const double omega = -2.0 * atan2(num, den);
        V3 acc = vscale(omega, n);
        for (int i = 0; i < 3; ++i) {
            const int j = (i + 1) % 3;
            const V3 e = vsub(vert(tr, j), vert(tr, i));
            const double L = sqrt(vdot(e, e));
            const V3 m = vscale(1.0 / L, vcross(e, n));   // outward in the face's plane
            const double s = R[i] + R[j];
            const double lg = log((s + L) / (s - L));
            acc = V3{acc.x + lg * m.x, acc.y + lg * m.y, acc.z + lg * m.z};
        }
        bx += tr.c * acc.x;
        by += tr.c * acc.y;
        bz += tr.c * acc.z;
    }
    float* o = out + 3 * idx;
    o[0] = (float)bx;
    o[1] = (float)by;
    o[2] = (float)bz;
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
    HeadTris T{};
    BPM_TRY(pole_triangles(G, &T));
    BPM_CK(cudaSetDevice(ctx->device));
    const size_t count = (size_t)nx * ny * nz;
    float* dst = B_T;
    if (!on_device) {
        cudaError_t e = cudaMallocAsync(&dst, count * 3 * sizeof(float), ctx->stream);
        if (e != cudaSuccess) {
            set_error("head-field buffer: %s", cudaGetErrorString(e));
            return BPM_ERR_OOM;
        }
    }
    const int threads = 256;
    k_head_field<<<(unsigned)((count + threads - 1) / threads), threads, 0, ctx->stream>>>(
        T, nx, ny, nz, h_nm, origin_nm[0], origin_nm[1], origin_nm[2], dst);
    cudaError_t e = cudaGetLastError();
    if (!on_device) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B_T, dst, count * 3 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        cudaFreeAsync(dst, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    if (e != cudaSuccess) {
        set_error("head-field solve: %s", cudaGetErrorString(e));
        return BPM_ERR_CUDA;
    }
    return BPM_OK;
}
