// One-time FP64 assembly of an island's operators on the GPU.
//
// P1 tetrahedral FEM (Sec. II.A: finite-element micromagnetics of the island;
// the discretisation itself is the textbook one): lumped nodal volumes, nodal
// Ms/Ku, the exchange stiffness K_ij = sum_t A_t vol_t grad(phi_i).grad(phi_j)
// and the exchange operator S = 2 K / (Ms V).  Demagnetising field by the
// hybrid FEM/BEM method (Sec. II.A) in the Fredkin-Koehler form:
//   u1: Neumann Poisson problem with source div(M) (zero-mean gauge),
//   u2 = (D + diag(Omega/4pi - 1)) u1 on the boundary, D the double-layer
//        matrix of Lindholm's closed-form weights for linear densities,
//   u2 harmonic inside (Dirichlet problem),
//   H = -grad(u1 + u2) per tet, lumped to the nodes.
// The map M -> H is applied to all 3n unit vectors at once: the Poisson
// problems are solved by Jacobi-preconditioned CG batched over the 3n
// right-hand sides (row-major [n][3n] blocks, one thread per entry, per-column
// reductions in a fixed order so that results are bit-reproducible).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <map>
#include <array>

#include "bpm_internal.cuh"

namespace bpm {

namespace {

struct DevPool {
    std::vector<void*> ptrs;
    ~DevPool() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    int alloc(T** p, size_t count, bool zero = true) {
        void* q = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T));
        if (e != cudaSuccess) {
            set_error("device allocation of %zu bytes failed: %s", count * sizeof(T),
                      cudaGetErrorString(e));
            return BPM_ERR_OOM;
        }
        ptrs.push_back(q);
        if (zero) {
            e = cudaMemset(q, 0, count * sizeof(T));
            if (e != cudaSuccess) {
                set_error("cudaMemset failed: %s", cudaGetErrorString(e));
                return BPM_ERR_CUDA;
            }
        }
        *p = static_cast<T*>(q);
        return BPM_OK;
    }
};

template <class T>
int upload(DevPool& pool, T** dst, const std::vector<T>& src) {
    BPM_TRY(pool.alloc(dst, src.size(), false));
    BPM_CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return BPM_OK;
}

// ---------------------------------------------------------------- vectors
struct V3 {
    double x, y, z;
};
__host__ __device__ inline V3 mk(double x, double y, double z) { return V3{x, y, z}; }
__host__ __device__ inline V3 sub(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ inline V3 add(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ inline V3 scl(V3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
__host__ __device__ inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline V3 cross(V3 a, V3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double nrm(V3 a) { return sqrt(dot(a, a)); }
__host__ __device__ inline V3 ld3(const double* p) { return mk(p[0], p[1], p[2]); }

// ---------------------------------------------------------------- FEM kernels
__global__ void k_tet_geom(int nt, const double* __restrict__ xyz, const int* __restrict__ tets,
                           double* __restrict__ vol, double* __restrict__ grads) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    V3 x0 = ld3(xyz + 3 * tets[4 * t + 0]);
    V3 e1 = sub(ld3(xyz + 3 * tets[4 * t + 1]), x0);
    V3 e2 = sub(ld3(xyz + 3 * tets[4 * t + 2]), x0);
    V3 e3 = sub(ld3(xyz + 3 * tets[4 * t + 3]), x0);
    V3 c23 = cross(e2, e3), c31 = cross(e3, e1), c12 = cross(e1, e2);
    double det = dot(e1, c23);
    // rows of J^{-1} (J = [e1 e2 e3]) are the gradients of phi_1..phi_3
    V3 g1 = scl(c23, 1.0 / det), g2 = scl(c31, 1.0 / det), g3 = scl(c12, 1.0 / det);
    V3 g0 = scl(add(add(g1, g2), g3), -1.0);
    vol[t] = fabs(det) / 6.0;
    double* g = grads + 12 * t;
    V3 gs[4] = {g0, g1, g2, g3};
    for (int a = 0; a < 4; ++a) {
        g[3 * a + 0] = gs[a].x;
        g[3 * a + 1] = gs[a].y;
        g[3 * a + 2] = gs[a].z;
    }
}

__device__ inline int local_index(const int* tet, int node) {
    for (int a = 0; a < 4; ++a)
        if (tet[a] == node) return a;
    return 0;
}

__device__ inline int find_col(const int* __restrict__ col, int lo, int hi, int j) {
    for (int e = lo; e < hi; ++e)
        if (col[e] == j) return e;
    return -1;
}

__global__ void k_node_lumped(int n, const int* __restrict__ n2t_ptr, const int* __restrict__ n2t,
                              const int* __restrict__ region, const double* __restrict__ vol,
                              const double* __restrict__ mat_Ms, const double* __restrict__ mat_Ku,
                              double* __restrict__ V, double* __restrict__ Ms, double* __restrict__ Ku) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 0, ms = 0, ku = 0;
    for (int e = n2t_ptr[i]; e < n2t_ptr[i + 1]; ++e) {
        int t = n2t[e];
        double q = 0.25 * vol[t];
        v += q;
        ms += q * mat_Ms[region[t]];
        ku += q * mat_Ku[region[t]];
    }
    V[i] = v;
    Ms[i] = ms / v;
    Ku[i] = ku / v;
}

__global__ void k_csr_values(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const int* __restrict__ n2t_ptr, const int* __restrict__ n2t,
                             const int* __restrict__ tets, const int* __restrict__ region,
                             const double* __restrict__ mat_A, const double* __restrict__ vol,
                             const double* __restrict__ grads, double* __restrict__ KA,
                             double* __restrict__ KL) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = n2t_ptr[i]; e < n2t_ptr[i + 1]; ++e) {
        int t = n2t[e];
        const int* tt = tets + 4 * t;
        int a = local_index(tt, i);
        const double* g = grads + 12 * t;
        for (int b = 0; b < 4; ++b) {
            int pos = find_col(col, rowptr[i], rowptr[i + 1], tt[b]);
            if (pos < 0) continue;
            double gg = g[3 * a] * g[3 * b] + g[3 * a + 1] * g[3 * b + 1] + g[3 * a + 2] * g[3 * b + 2];
            KL[pos] += vol[t] * gg;
            KA[pos] += mat_A[region[t]] * vol[t] * gg;
        }
    }
}

// exchange operator, difference form: c_ij = -2e18 K_A,ij / (Ms_i V_i) for j != i
// (nm -> m: K carries 1e-9, V carries 1e-27)
__global__ void k_exchange_values(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                  const double* __restrict__ KA, const double* __restrict__ V,
                                  const double* __restrict__ Ms, float* __restrict__ c) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = -2.0e18 / (Ms[i] * V[i]);
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) c[e] = (col[e] == i) ? 0.f : (float)(s * KA[e]);
}

// the same values in FP64, kept for the plain FP64 form
__global__ void k_exchange_values64(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                    const double* __restrict__ KA, const double* __restrict__ V,
                                    const double* __restrict__ Ms, double* __restrict__ c) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = -2.0e18 / (Ms[i] * V[i]);
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) c[e] = (col[e] == i) ? 0.0 : s * KA[e];
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0;
    int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) s += red[k];
    return s;
}

// Largest eigenvalue of S = D K_A (D = 2e18/(Ms V)) by power iteration on the
// similar symmetric matrix D^1/2 K_A D^1/2; one block, Rayleigh quotient.
__global__ void k_power_iteration(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                  const double* __restrict__ KA, const double* __restrict__ V,
                                  const double* __restrict__ Ms, double* x, double* y, int iters,
                                  double* lam_out) {
    __shared__ double red[32];
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        x[i] = ((i & 1) ? 1.0 : -1.0) + 0.3 * sin(0.7 * i);
    __syncthreads();
    double lam = 0;
    for (int it = 0; it < iters; ++it) {
        double nn = 0, xy = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double di = sqrt(2.0e18 / (Ms[i] * V[i]));
            double s = 0;
            for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                int j = col[e];
                s += KA[e] * sqrt(2.0e18 / (Ms[j] * V[j])) * x[j];
            }
            y[i] = di * s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            nn += y[i] * y[i];
            xy += x[i] * y[i];
        }
        double xx = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) xx += x[i] * x[i];
        nn = block_sum(nn, red);
        xy = block_sum(xy, red);
        xx = block_sum(xx, red);
        lam = xy / xx;
        double inv = 1.0 / sqrt(nn);
        for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = y[i] * inv;
        __syncthreads();
    }
    if (threadIdx.x == 0) *lam_out = lam;
}

// R [n][3n]: (R M)_i = int M . grad(phi_i) for nodal P1 M; column c*n + k
__global__ void k_rhs(int n, const int* __restrict__ n2t_ptr, const int* __restrict__ n2t,
                      const int* __restrict__ tets, const double* __restrict__ vol,
                      const double* __restrict__ grads, double* __restrict__ R) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    size_t ncol = 3 * (size_t)n;
    for (int e = n2t_ptr[i]; e < n2t_ptr[i + 1]; ++e) {
        int t = n2t[e];
        const int* tt = tets + 4 * t;
        int a = local_index(tt, i);
        const double* g = grads + 12 * t;
        double q = 0.25 * vol[t];
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 3; ++c) R[i * ncol + (size_t)c * n + tt[b]] += q * g[3 * a + c];
    }
}

// ---------------------------------------------------------------- batched CG
// Y[i][c] = sum_e val_e X[col_e][c]; with mask: rows and columns outside the mask are zero
__global__ void k_spmm(int n, int ncol, const int* __restrict__ rowptr, const int* __restrict__ col,
                       const double* __restrict__ val, const unsigned char* __restrict__ mask,
                       const double* __restrict__ X, double* __restrict__ Y) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (c >= ncol) return;
    double s = 0;
    if (!mask || mask[i]) {
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            int j = col[e];
            if (mask && !mask[j]) continue;
            s += val[e] * X[(size_t)j * ncol + c];
        }
    }
    Y[(size_t)i * ncol + c] = s;
}

__global__ void k_coldot(int n, int ncol, const double* __restrict__ X, const double* __restrict__ Y,
                         double* __restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    double s = 0;
    for (int i = 0; i < n; ++i) s += X[(size_t)i * ncol + c] * Y[(size_t)i * ncol + c];
    out[c] = s;
}

__global__ void k_cg_init(int n, int ncol, const double* __restrict__ b, const double* __restrict__ dinv,
                          double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                          double* __restrict__ p) {
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * ncol) return;
    int i = (int)(k / ncol);
    x[k] = 0;
    r[k] = b[k];
    z[k] = dinv[i] * b[k];
    p[k] = z[k];
}

__global__ void k_cg_xr(int n, int ncol, const double* __restrict__ rz, const double* __restrict__ pq,
                        const double* __restrict__ dinv, const double* __restrict__ p,
                        const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                        double* __restrict__ z) {
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * ncol) return;
    int i = (int)(k / ncol), c = (int)(k % ncol);
    double a = pq[c] > 0 ? rz[c] / pq[c] : 0.0;
    x[k] += a * p[k];
    double rv = r[k] - a * q[k];
    r[k] = rv;
    z[k] = dinv[i] * rv;
}

__global__ void k_cg_p(int n, int ncol, const double* __restrict__ rz_new, double* __restrict__ rz_old,
                       const double* __restrict__ z, double* __restrict__ p) {
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * ncol) return;
    int c = (int)(k % ncol);
    double b = rz_old[c] > 0 ? rz_new[c] / rz_old[c] : 0.0;
    p[k] = z[k] + b * p[k];
}

__global__ void k_copy_vec(int ncol, const double* __restrict__ a, double* __restrict__ b) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncol) b[c] = a[c];
}

__global__ void k_max_ratio(int ncol, const double* __restrict__ rr, const double* __restrict__ bb,
                            double* __restrict__ out) {
    __shared__ double red[32];
    double m = 0;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        double v = bb[c] > 0 ? sqrt(rr[c] / bb[c]) : 0.0;
        if (!(v == v)) v = 1e300;  // NaN propagates as "not converged"
        m = fmax(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s = fmax(s, red[k]);
        *out = s;
    }
}

__global__ void k_col_mean_sub(int n, int ncol, double* __restrict__ X) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    double s = 0;
    for (int i = 0; i < n; ++i) s += X[(size_t)i * ncol + c];
    s /= n;
    for (int i = 0; i < n; ++i) X[(size_t)i * ncol + c] -= s;
}

__global__ void k_masked_scale(int n, int ncol, const unsigned char* __restrict__ mask, double s,
                               double* __restrict__ X) {
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * ncol) return;
    int i = (int)(k / ncol);
    X[k] = mask[i] ? s * X[k] : 0.0;
}

int pcg(cudaStream_t st, DevPool& pool, int n, int ncol, const int* rowptr, const int* col,
        const double* val, const unsigned char* mask, const double* dinv, const double* b,
        double* x, double tol, int maxit, int* iters_out, double* resid_out) {
    size_t N = (size_t)n * ncol;
    double *r, *z, *p, *q, *rz, *rzn, *pq, *bb, *rr, *mx;
    BPM_TRY(pool.alloc(&r, N, false));
    BPM_TRY(pool.alloc(&z, N, false));
    BPM_TRY(pool.alloc(&p, N, false));
    BPM_TRY(pool.alloc(&q, N, false));
    BPM_TRY(pool.alloc(&rz, ncol));
    BPM_TRY(pool.alloc(&rzn, ncol));
    BPM_TRY(pool.alloc(&pq, ncol));
    BPM_TRY(pool.alloc(&bb, ncol));
    BPM_TRY(pool.alloc(&rr, ncol));
    BPM_TRY(pool.alloc(&mx, 1));
    const int T = 256;
    unsigned gN = (unsigned)((N + T - 1) / T), gC = (unsigned)((ncol + T - 1) / T);
    dim3 gS((ncol + 127) / 128, n);
    k_cg_init<<<gN, T, 0, st>>>(n, ncol, b, dinv, x, r, z, p);
    k_coldot<<<gC, T, 0, st>>>(n, ncol, r, z, rz);
    k_coldot<<<gC, T, 0, st>>>(n, ncol, b, b, bb);
    BPM_CK(cudaGetLastError());
    double res = 1.0;
    int it = 0;
    for (it = 1; it <= maxit; ++it) {
        k_spmm<<<gS, 128, 0, st>>>(n, ncol, rowptr, col, val, mask, p, q);
        k_coldot<<<gC, T, 0, st>>>(n, ncol, p, q, pq);
        k_cg_xr<<<gN, T, 0, st>>>(n, ncol, rz, pq, dinv, p, q, x, r, z);
        k_coldot<<<gC, T, 0, st>>>(n, ncol, r, z, rzn);
        k_cg_p<<<gN, T, 0, st>>>(n, ncol, rzn, rz, z, p);
        k_copy_vec<<<gC, T, 0, st>>>(ncol, rzn, rz);
        if (it % 16 == 0 || it == maxit) {
            k_coldot<<<gC, T, 0, st>>>(n, ncol, r, r, rr);
            k_max_ratio<<<1, 1024, 0, st>>>(ncol, rr, bb, mx);
            BPM_CK(cudaGetLastError());
            BPM_CK(cudaMemcpyAsync(&res, mx, sizeof(double), cudaMemcpyDeviceToHost, st));
            BPM_CK(cudaStreamSynchronize(st));
            if (!(res < 1e300)) {
                set_error("CG produced a non-finite residual");
                return BPM_ERR_NONFINITE;
            }
            if (res < tol) break;
        }
    }
    *iters_out = std::min(it, maxit);
    *resid_out = res;
    if (res >= tol) {
        set_error("CG did not converge: relative residual %.3e after %d iterations", res, maxit);
        return BPM_ERR_UNSTABLE;
    }
    return BPM_OK;
}

// ---------------------------------------------------------------- BEM
// signed solid angle of triangle (r1, r2, r3) seen from the origin (van Oosterom & Strackee)
__device__ double solid_angle(V3 r1, V3 r2, V3 r3) {
    double l1 = nrm(r1), l2 = nrm(r2), l3 = nrm(r3);
    double num = dot(r1, cross(r2, r3));
    double den = l1 * l2 * l3 + dot(r1, r2) * l3 + dot(r1, r3) * l2 + dot(r2, r3) * l1;
    return 2.0 * atan2(num, den);
}

// w_k = int_T phi_k(y) n.(y - x)/|y - x|^3 dS, Lindholm's closed form (see header of this file)
__device__ void lindholm(V3 x, const V3 y[3], double w[3]) {
    V3 rho[3], xi[3];
    double s[3], lr[3];
    for (int k = 0; k < 3; ++k) {
        rho[k] = sub(y[k], x);
        lr[k] = nrm(rho[k]);
        V3 e = sub(y[(k + 1) % 3], y[k]);
        s[k] = nrm(e);
        xi[k] = scl(e, 1.0 / s[k]);
    }
    V3 cr = cross(sub(y[1], y[0]), sub(y[2], y[0]));
    double two_area = nrm(cr);
    V3 n = scl(cr, 1.0 / two_area);
    double zeta = dot(n, rho[0]);
    double eta[3], P[3];
    for (int k = 0; k < 3; ++k) {
        eta[k] = dot(cross(n, xi[k]), rho[k]);
        double ls = lr[k] + lr[(k + 1) % 3];
        P[k] = log((ls + s[k]) / (ls - s[k]));
    }
    double om = solid_angle(rho[0], rho[1], rho[2]);
    for (int k = 0; k < 3; ++k) {
        int k1 = (k + 1) % 3;
        double gp = 0;
        for (int j = 0; j < 3; ++j) gp += dot(xi[k1], xi[j]) * P[j];
        w[k] = s[k1] / two_area * (-eta[k1] * om + zeta * gp);
    }
}

__global__ void k_interior_angles(int nb, const int* __restrict__ bnodes, const int* __restrict__ n2t_ptr,
                                  const int* __restrict__ n2t, const int* __restrict__ tets,
                                  const double* __restrict__ xyz, double* __restrict__ omega) {
    int ib = blockIdx.x * blockDim.x + threadIdx.x;
    if (ib >= nb) return;
    int i = bnodes[ib];
    V3 x = ld3(xyz + 3 * i);
    double s = 0;
    for (int e = n2t_ptr[i]; e < n2t_ptr[i + 1]; ++e) {
        const int* tt = tets + 4 * n2t[e];
        V3 r[3];
        int k = 0;
        for (int a = 0; a < 4; ++a)
            if (tt[a] != i) r[k++] = sub(ld3(xyz + 3 * tt[a]), x);
        s += fabs(solid_angle(r[0], r[1], r[2]));
    }
    omega[ib] = s;
}

// Bmat[ib][jb] = D_ij + delta_ij (Omega_i/4pi - 1),
// D_ij = -(1/4pi) sum over boundary faces T containing node j (not node i) of w_j(x_i; T)
__global__ void k_bem_matrix(int nb, const int* __restrict__ bnodes, const double* __restrict__ xyz,
                             const int* __restrict__ faces, const int* __restrict__ b2f_ptr,
                             const int* __restrict__ b2f, const double* __restrict__ omega,
                             double* __restrict__ Bmat) {
    int jb = blockIdx.x * blockDim.x + threadIdx.x;
    int ib = blockIdx.y;
    if (jb >= nb) return;
    int i = bnodes[ib], j = bnodes[jb];
    V3 x = ld3(xyz + 3 * i);
    double s = 0;
    for (int e = b2f_ptr[jb]; e < b2f_ptr[jb + 1]; ++e) {
        const int* f = faces + 3 * b2f[e];
        if (f[0] == i || f[1] == i || f[2] == i) continue;  // x_i in the face plane: weight 0
        V3 y[3] = {ld3(xyz + 3 * f[0]), ld3(xyz + 3 * f[1]), ld3(xyz + 3 * f[2])};
        double w[3];
        lindholm(x, y, w);
        int loc = (f[0] == j) ? 0 : ((f[1] == j) ? 1 : 2);
        s += w[loc];
    }
    double v = -s / (4.0 * M_PI);
    if (ib == jb) v += omega[ib] / (4.0 * M_PI) - 1.0;
    Bmat[(size_t)ib * nb + jb] = v;
}

__global__ void k_gather_rows(int nb, int ncol, const int* __restrict__ rows, const double* __restrict__ src,
                              double* __restrict__ dst) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int ib = blockIdx.y;
    if (c >= ncol) return;
    dst[(size_t)ib * ncol + c] = src[(size_t)rows[ib] * ncol + c];
}

__global__ void k_scatter_rows(int nb, int ncol, const int* __restrict__ rows, const double* __restrict__ src,
                               double* __restrict__ dst) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int ib = blockIdx.y;
    if (c >= ncol) return;
    dst[(size_t)rows[ib] * ncol + c] = src[(size_t)ib * ncol + c];
}

// C[M][N] = A[M][K] B[K][N] (row-major, FP64), 32x32 tiles
__global__ void k_dgemm(int M, int N, int K, const double* __restrict__ A, const double* __restrict__ B,
                        double* __restrict__ C) {
    __shared__ double As[32][33], Bs[32][33];
    int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    int row0 = blockIdx.y * 32, col = blockIdx.x * 32 + tx;
    double acc[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            int gr = row0 + r, gk = k0 + tx;
            As[r][tx] = (gr < M && gk < K) ? A[(size_t)gr * K + gk] : 0.0;
            int bk = k0 + r;
            Bs[r][tx] = (bk < K && col < N) ? B[(size_t)bk * N + col] : 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk < 32; ++kk) {
            double bv = Bs[kk][tx];
            for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][kk] * bv;
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        int gr = row0 + ty + 8 * q;
        if (gr < M && col < N) C[(size_t)gr * N + col] = acc[q];
    }
}

__global__ void k_add3(size_t N, const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ c, double* __restrict__ out) {
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) out[k] = a[k] + b[k] + c[k];
}

// P_c[e] = (1/V_i) sum_{t ni i, k} (vol_t / 4) grad(phi_k)|_t [c] for CSR entry e = (i, k)
__global__ void k_proj_values(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                              const int* __restrict__ n2t_ptr, const int* __restrict__ n2t,
                              const int* __restrict__ tets, const double* __restrict__ vol,
                              const double* __restrict__ grads, const double* __restrict__ V, int nnz,
                              double* __restrict__ P) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = n2t_ptr[i]; e < n2t_ptr[i + 1]; ++e) {
        int t = n2t[e];
        const int* tt = tets + 4 * t;
        const double* g = grads + 12 * t;
        double q = 0.25 * vol[t] / V[i];
        for (int b = 0; b < 4; ++b) {
            int pos = find_col(col, rowptr[i], rowptr[i + 1], tt[b]);
            if (pos < 0) continue;
            for (int c = 0; c < 3; ++c) P[(size_t)c * nnz + pos] += q * g[3 * b + c];
        }
    }
}

// N64[(c n + i)][col] = sum_e P_c[e] U[col_e][col]   (H = -N M with u = U M)
__global__ void k_demag_rows(int n, int ncol, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const double* __restrict__ P, int nnz, const double* __restrict__ U,
                             double* __restrict__ N64) {
    int cc = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (cc >= ncol) return;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        double u = U[(size_t)col[e] * ncol + cc];
        s0 += P[e] * u;
        s1 += P[(size_t)nnz + e] * u;
        s2 += P[2 * (size_t)nnz + e] * u;
    }
    N64[((size_t)0 * n + i) * ncol + cc] = s0;
    N64[((size_t)1 * n + i) * ncol + cc] = s1;
    N64[((size_t)2 * n + i) * ncol + cc] = s2;
}

// padded kernel operand [K][K]: W[r][q] = -mu0 1e6 N[(c n + i)][(c' n + k)], r = c n_pad + i,
// q = c' n_pad + k; zero on padding nodes and on rows/columns from 3 n_pad to K
__global__ void k_demag_convert(int n, int n_pad, int K, const double* __restrict__ N64, float* __restrict__ W32,
                                __nv_bfloat16* __restrict__ Whi, __nv_bfloat16* __restrict__ Wlo) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (q >= K) return;
    int c = r / n_pad, i = r % n_pad, c2 = q / n_pad, k = q % n_pad;
    double v = 0;
    if (c < 3 && c2 < 3 && i < n && k < n) v = -kMu0 * 1e6 * N64[((size_t)c * n + i) * (3 * (size_t)n) + (size_t)c2 * n + k];
    size_t o = (size_t)r * K + q;
    W32[o] = (float)v;
    __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
    Whi[o] = hi;
    Wlo[o] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
}

}  // namespace

void free_mesh(Mesh* M) {
    if (!M) return;
    cudaFree(M->node_pos);
    cudaFree(M->node_mat);
    cudaFree(M->sell_off);
    cudaFree(M->sell_ent);
    cudaFree(M->sell_il);
    cudaFree(M->N32);
    cudaFree(M->Nhi);
    cudaFree(M->Nlo);
    cudaFree(M->N64);
    cudaFree(M->csr_rowptr);
    cudaFree(M->csr_col);
    cudaFree(M->csr_c64);
    cudaFree(M->node64);
    cudaFree(M->mat64);
    delete M;
}

int assemble_mesh(bpm_ctx* ctx, Mesh* M, const double* xyz, const int32_t* tets_in, int32_t nt,
                  const int32_t* region, const bpm_region_mat* mats, int32_t nreg, uint32_t flags) {
    const int n = M->n;
    cudaStream_t st = ctx->stream;
    // ---------------- host topology ----------------
    std::vector<int> tets(tets_in, tets_in + 4 * (size_t)nt);
    for (int t = 0; t < nt; ++t) {
        for (int a = 0; a < 4; ++a)
            if (tets[4 * t + a] < 0 || tets[4 * t + a] >= n) {
                set_error("tet %d references node %d outside [0, %d)", t, tets[4 * t + a], n);
                return BPM_ERR_ARG;
            }
        if (region[t] < 0 || region[t] >= nreg) {
            set_error("tet %d has region %d outside [0, %d)", t, region[t], nreg);
            return BPM_ERR_ARG;
        }
        V3 x0 = ld3(xyz + 3 * tets[4 * t]);
        V3 e1 = sub(ld3(xyz + 3 * tets[4 * t + 1]), x0), e2 = sub(ld3(xyz + 3 * tets[4 * t + 2]), x0),
           e3 = sub(ld3(xyz + 3 * tets[4 * t + 3]), x0);
        double det = dot(e1, cross(e2, e3));
        double h = std::max(nrm(e1), std::max(nrm(e2), nrm(e3)));
        if (!(fabs(det) > 1e-10 * h * h * h)) {
            set_error("tet %d is degenerate", t);
            return BPM_ERR_ARG;
        }
    }
    // node -> tets
    std::vector<int> n2t_ptr(n + 1, 0), n2t(4 * (size_t)nt);
    for (int k = 0; k < 4 * nt; ++k) n2t_ptr[tets[k] + 1]++;
    for (int i = 0; i < n; ++i) n2t_ptr[i + 1] += n2t_ptr[i];
    {
        std::vector<int> fill(n2t_ptr.begin(), n2t_ptr.end() - 1);
        for (int t = 0; t < nt; ++t)
            for (int a = 0; a < 4; ++a) n2t[fill[tets[4 * t + a]]++] = t;
    }
    for (int i = 0; i < n; ++i)
        if (n2t_ptr[i + 1] == n2t_ptr[i]) {
            set_error("node %d belongs to no tetrahedron", i);
            return BPM_ERR_ARG;
        }
    // CSR pattern (sorted, incl. diagonal)
    std::vector<int>& rowptr = M->rowptr;
    std::vector<int>& col = M->col;
    rowptr.assign(n + 1, 0);
    col.clear();
    {
        std::vector<int> nb;
        for (int i = 0; i < n; ++i) {
            nb.clear();
            for (int e = n2t_ptr[i]; e < n2t_ptr[i + 1]; ++e)
                for (int a = 0; a < 4; ++a) nb.push_back(tets[4 * n2t[e] + a]);
            std::sort(nb.begin(), nb.end());
            nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
            col.insert(col.end(), nb.begin(), nb.end());
            rowptr[i + 1] = (int)col.size();
        }
    }
    const int nnz = (int)col.size();
    // boundary faces: faces of exactly one tet, oriented outward
    std::map<std::array<int, 3>, std::array<int, 5>> fmap;  // key -> {count, a, b, c, opposite}
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 4; ++k) {
            int f[3], q = 0;
            for (int a = 0; a < 4; ++a)
                if (a != k) f[q++] = tets[4 * t + a];
            std::array<int, 3> key{f[0], f[1], f[2]};
            std::sort(key.begin(), key.end());
            auto it = fmap.find(key);
            if (it == fmap.end())
                fmap[key] = {1, f[0], f[1], f[2], tets[4 * t + k]};
            else
                it->second[0]++;
        }
    std::vector<int> faces;
    for (auto& kv : fmap) {
        if (kv.second[0] != 1) continue;
        int a = kv.second[1], b = kv.second[2], c = kv.second[3], d = kv.second[4];
        V3 ya = ld3(xyz + 3 * a);
        V3 nrmv = cross(sub(ld3(xyz + 3 * b), ya), sub(ld3(xyz + 3 * c), ya));
        if (dot(nrmv, sub(ld3(xyz + 3 * d), ya)) > 0) std::swap(b, c);
        faces.push_back(a);
        faces.push_back(b);
        faces.push_back(c);
    }
    const int nf = (int)faces.size() / 3;
    std::vector<int> bnodes(faces.begin(), faces.end());
    std::sort(bnodes.begin(), bnodes.end());
    bnodes.erase(std::unique(bnodes.begin(), bnodes.end()), bnodes.end());
    const int nb = (int)bnodes.size();
    std::vector<int> bidx(n, -1);
    for (int k = 0; k < nb; ++k) bidx[bnodes[k]] = k;
    std::vector<int> b2f_ptr(nb + 1, 0), b2f(3 * (size_t)nf);
    for (int k = 0; k < 3 * nf; ++k) b2f_ptr[bidx[faces[k]] + 1]++;
    for (int k = 0; k < nb; ++k) b2f_ptr[k + 1] += b2f_ptr[k];
    {
        std::vector<int> fill(b2f_ptr.begin(), b2f_ptr.end() - 1);
        for (int f = 0; f < nf; ++f)
            for (int a = 0; a < 3; ++a) b2f[fill[bidx[faces[3 * f + a]]]++] = f;
    }
    std::vector<unsigned char> interior(n, 1);
    for (int k = 0; k < nb; ++k) interior[bnodes[k]] = 0;
    std::vector<double> mat_Ms(nreg), mat_Ku(nreg), mat_A(nreg);
    for (int r = 0; r < nreg; ++r) {
        mat_Ms[r] = mats[r].Ms_A_per_m;
        mat_Ku[r] = mats[r].Ku_J_per_m3;
        mat_A[r] = mats[r].A_J_per_m;
        if (!(mat_Ms[r] > 0)) {
            set_error("region %d has Ms <= 0", r);
            return BPM_ERR_ARG;
        }
    }

    // ---------------- device assembly ----------------
    DevPool pool;
    double *d_xyz, *d_vol, *d_grads, *d_V, *d_Ms, *d_Ku, *d_KA, *d_KL, *d_mMs, *d_mKu, *d_mA;
    int *d_tets, *d_reg, *d_n2tp, *d_n2t, *d_rowptr, *d_col, *d_bnodes, *d_faces, *d_b2fp, *d_b2f;
    unsigned char* d_int;
    std::vector<double> xyzv(xyz, xyz + 3 * (size_t)n);
    std::vector<int> regv(region, region + nt);
    BPM_TRY(upload(pool, &d_xyz, xyzv));
    BPM_TRY(upload(pool, &d_tets, tets));
    BPM_TRY(upload(pool, &d_reg, regv));
    BPM_TRY(upload(pool, &d_n2tp, n2t_ptr));
    BPM_TRY(upload(pool, &d_n2t, n2t));
    BPM_TRY(upload(pool, &d_rowptr, rowptr));
    BPM_TRY(upload(pool, &d_col, col));
    BPM_TRY(upload(pool, &d_bnodes, bnodes));
    BPM_TRY(upload(pool, &d_faces, faces));
    BPM_TRY(upload(pool, &d_b2fp, b2f_ptr));
    BPM_TRY(upload(pool, &d_b2f, b2f));
    BPM_TRY(upload(pool, &d_int, interior));
    BPM_TRY(upload(pool, &d_mMs, mat_Ms));
    BPM_TRY(upload(pool, &d_mKu, mat_Ku));
    BPM_TRY(upload(pool, &d_mA, mat_A));
    BPM_TRY(pool.alloc(&d_vol, nt));
    BPM_TRY(pool.alloc(&d_grads, 12 * (size_t)nt));
    BPM_TRY(pool.alloc(&d_V, n));
    BPM_TRY(pool.alloc(&d_Ms, n));
    BPM_TRY(pool.alloc(&d_Ku, n));
    BPM_TRY(pool.alloc(&d_KA, nnz));
    BPM_TRY(pool.alloc(&d_KL, nnz));
    const int T = 256;
    k_tet_geom<<<(nt + T - 1) / T, T, 0, st>>>(nt, d_xyz, d_tets, d_vol, d_grads);
    k_node_lumped<<<(n + T - 1) / T, T, 0, st>>>(n, d_n2tp, d_n2t, d_reg, d_vol, d_mMs, d_mKu, d_V, d_Ms, d_Ku);
    k_csr_values<<<(n + T - 1) / T, T, 0, st>>>(n, d_rowptr, d_col, d_n2tp, d_n2t, d_tets, d_reg, d_mA,
                                                 d_vol, d_grads, d_KA, d_KL);
    BPM_CK(cudaGetLastError());
    // exchange operator values (FP32) and lambda_max
    float* d_c;
    BPM_TRY(pool.alloc(&d_c, nnz));
    k_exchange_values<<<(n + T - 1) / T, T, 0, st>>>(n, d_rowptr, d_col, d_KA, d_V, d_Ms, d_c);
    BPM_CK(cudaMalloc(&M->csr_rowptr, (n + 1) * sizeof(int)));
    BPM_CK(cudaMalloc(&M->csr_col, nnz * sizeof(int)));
    BPM_CK(cudaMalloc(&M->csr_c64, nnz * sizeof(double)));
    BPM_CK(cudaMemcpyAsync(M->csr_rowptr, d_rowptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToDevice, st));
    BPM_CK(cudaMemcpyAsync(M->csr_col, d_col, nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
    k_exchange_values64<<<(n + T - 1) / T, T, 0, st>>>(n, d_rowptr, d_col, d_KA, d_V, d_Ms, M->csr_c64);
    double *d_px, *d_py, *d_lam;
    BPM_TRY(pool.alloc(&d_px, n));
    BPM_TRY(pool.alloc(&d_py, n));
    BPM_TRY(pool.alloc(&d_lam, 1));
    k_power_iteration<<<1, 1024, 0, st>>>(n, d_rowptr, d_col, d_KA, d_V, d_Ms, d_px, d_py, 1500, d_lam);
    BPM_CK(cudaGetLastError());
    M->exch_val.resize(nnz);
    M->V.resize(n);
    M->Ms.resize(n);
    M->Ku.resize(n);
    double lam = 0;
    BPM_CK(cudaMemcpyAsync(M->exch_val.data(), d_c, nnz * sizeof(float), cudaMemcpyDeviceToHost, st));
    BPM_CK(cudaMemcpyAsync(M->V.data(), d_V, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    BPM_CK(cudaMemcpyAsync(M->Ms.data(), d_Ms, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    BPM_CK(cudaMemcpyAsync(M->Ku.data(), d_Ku, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    BPM_CK(cudaMemcpyAsync(&lam, d_lam, sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<double> KLh(nnz);
    BPM_CK(cudaMemcpyAsync(KLh.data(), d_KL, nnz * sizeof(double), cudaMemcpyDeviceToHost, st));
    BPM_CK(cudaStreamSynchronize(st));

    // ---------------- Fredkin-Koehler demag ----------------
    const int ncol = 3 * n;
    const size_t NN = (size_t)n * ncol;
    double *d_R, *d_U1, *d_dinvN, *d_dinvD;
    BPM_TRY(pool.alloc(&d_R, NN));
    k_rhs<<<(n + T - 1) / T, T, 0, st>>>(n, d_n2tp, d_n2t, d_tets, d_vol, d_grads, d_R);
    BPM_CK(cudaGetLastError());
    std::vector<double> dinvN(n), dinvD(n);
    for (int i = 0; i < n; ++i) {
        double kii = 0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
            if (col[e] == i) kii = KLh[e];
        dinvN[i] = 1.0 / kii;
        dinvD[i] = interior[i] ? 1.0 / kii : 0.0;
    }
    BPM_TRY(upload(pool, &d_dinvN, dinvN));
    BPM_TRY(upload(pool, &d_dinvD, dinvD));
    BPM_TRY(pool.alloc(&d_U1, NN, false));
    int it1 = 0, it2 = 0;
    double res1 = 0, res2 = 0;
    BPM_TRY(pcg(st, pool, n, ncol, d_rowptr, d_col, d_KL, nullptr, d_dinvN, d_R, d_U1, 1e-12, 20000, &it1, &res1));
    k_col_mean_sub<<<(ncol + T - 1) / T, T, 0, st>>>(n, ncol, d_U1);
    // boundary values of u2
    double *d_omega, *d_Bmat, *d_U1B, *d_U2B, *d_U2e, *d_bD, *d_U2I;
    BPM_TRY(pool.alloc(&d_omega, nb));
    BPM_TRY(pool.alloc(&d_Bmat, (size_t)nb * nb, false));
    BPM_TRY(pool.alloc(&d_U1B, (size_t)nb * ncol, false));
    BPM_TRY(pool.alloc(&d_U2B, (size_t)nb * ncol, false));
    k_interior_angles<<<(nb + 127) / 128, 128, 0, st>>>(nb, d_bnodes, d_n2tp, d_n2t, d_tets, d_xyz, d_omega);
    k_bem_matrix<<<dim3((nb + 127) / 128, nb), 128, 0, st>>>(nb, d_bnodes, d_xyz, d_faces, d_b2fp, d_b2f,
                                                             d_omega, d_Bmat);
    k_gather_rows<<<dim3((ncol + 127) / 128, nb), 128, 0, st>>>(nb, ncol, d_bnodes, d_U1, d_U1B);
    k_dgemm<<<dim3((ncol + 31) / 32, (nb + 31) / 32), dim3(32, 8), 0, st>>>(nb, ncol, nb, d_Bmat, d_U1B, d_U2B);
    BPM_CK(cudaGetLastError());
    // harmonic extension: K_II u2_I = -K_IB u2_B
    BPM_TRY(pool.alloc(&d_U2e, NN));
    BPM_TRY(pool.alloc(&d_bD, NN, false));
    BPM_TRY(pool.alloc(&d_U2I, NN));
    k_scatter_rows<<<dim3((ncol + 127) / 128, nb), 128, 0, st>>>(nb, ncol, d_bnodes, d_U2B, d_U2e);
    k_spmm<<<dim3((ncol + 127) / 128, n), 128, 0, st>>>(n, ncol, d_rowptr, d_col, d_KL, nullptr, d_U2e, d_bD);
    k_masked_scale<<<(unsigned)((NN + T - 1) / T), T, 0, st>>>(n, ncol, d_int, -1.0, d_bD);
    BPM_CK(cudaGetLastError());
    if (nb < n)
        BPM_TRY(pcg(st, pool, n, ncol, d_rowptr, d_col, d_KL, d_int, d_dinvD, d_bD, d_U2I, 1e-12, 20000, &it2,
                    &res2));
    // u = u1 + u2 ; N = P u
    double *d_U, *d_P;
    BPM_TRY(pool.alloc(&d_U, NN, false));
    k_add3<<<(unsigned)((NN + T - 1) / T), T, 0, st>>>(NN, d_U1, d_U2e, d_U2I, d_U);
    BPM_TRY(pool.alloc(&d_P, 3 * (size_t)nnz));
    k_proj_values<<<(n + T - 1) / T, T, 0, st>>>(n, d_rowptr, d_col, d_n2tp, d_n2t, d_tets, d_vol, d_grads, d_V,
                                                 nnz, d_P);
    BPM_CK(cudaGetLastError());
    double* N64 = nullptr;
    BPM_CK(cudaMalloc(&N64, (size_t)ncol * ncol * sizeof(double)));
    M->N64 = N64;  // freed below unless kept
    k_demag_rows<<<dim3((ncol + 127) / 128, n), 128, 0, st>>>(n, ncol, d_rowptr, d_col, d_P, nnz, d_U, N64);
    const int K = M->K();
    BPM_CK(cudaMalloc(&M->N32, (size_t)K * K * sizeof(float)));
    BPM_CK(cudaMalloc(&M->Nhi, (size_t)K * K * sizeof(__nv_bfloat16)));
    BPM_CK(cudaMalloc(&M->Nlo, (size_t)K * K * sizeof(__nv_bfloat16)));
    k_demag_convert<<<dim3((K + 127) / 128, K), 128, 0, st>>>(n, M->n_pad, K, N64, M->N32, M->Nhi, M->Nlo);
    BPM_CK(cudaGetLastError());
    BPM_CK(cudaStreamSynchronize(st));
    if (!(flags & BPM_MESH_KEEP_F64)) {
        cudaFree(M->N64);
        M->N64 = nullptr;
    }

    // ---------------- node data and sliced-ELL exchange ----------------
    const int np = M->n_pad;
    double Vsum = 0;
    for (int i = 0; i < n; ++i) Vsum += M->V[i];
    std::vector<float4> pos(np, make_float4(0, 0, 0, 0)), nm(np, make_float4(0, 0, 0, 0));
    double an_max = 0, ms_max = 0;
    for (int i = 0; i < n; ++i) {
        pos[i] = make_float4((float)xyz[3 * i], (float)xyz[3 * i + 1], (float)xyz[3 * i + 2],
                             (float)(M->V[i] / Vsum));

        double an = 2.0 * M->Ku[i] / M->Ms[i];
        nm[i] = make_float4((float)an, (float)(M->Ms[i] * 1e-6), 0.f, 0.f);
        an_max = std::max(an_max, an);
        ms_max = std::max(ms_max, M->Ms[i]);
    }
    M->n_slices = np / 32;
    std::vector<int> off(M->n_slices + 1, 0);
    for (int s = 0; s < M->n_slices; ++s) {
        int w = 0;
        for (int l = 0; l < 32; ++l) {
            int i = 32 * s + l;
            if (i < n) w = std::max(w, rowptr[i + 1] - rowptr[i] - 1);
        }
        off[s + 1] = off[s] + 32 * w;
    }
    std::vector<int2> ent(std::max(1, off[M->n_slices]));
    for (int s = 0; s < M->n_slices; ++s) {
        int w = (off[s + 1] - off[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            int i = 32 * s + l;
            int q = 0;
            if (i < n)
                for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                    if (col[e] == i) continue;
                    float v = M->exch_val[e];
                    ent[off[s] + 32 * q + l] = make_int2(col[e], *reinterpret_cast<int*>(&v));
                    ++q;
                }
            for (; q < w; ++q) ent[off[s] + 32 * q + l] = make_int2(i < n ? i : 0, 0);
        }
    }
    std::vector<int2> ent_il(ent.size());
    for (size_t k = 0; k < ent.size(); ++k) {
        const int j = ent[k].x;
        ent_il[k] = make_int2(4 * ((j >> 5) * 96 * kIlIslands + (j & 31)), ent[k].y);
    }
    std::vector<NodeF64> node64(n);
    std::vector<double2> mat64(n);
    for (int i = 0; i < n; ++i) {
        node64[i] = NodeF64{xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], M->V[i] / Vsum};
        mat64[i] = make_double2(2.0 * M->Ku[i] / M->Ms[i], M->Ms[i]);
    }
    BPM_CK(cudaMalloc(&M->node64, n * sizeof(NodeF64)));
    BPM_CK(cudaMalloc(&M->mat64, n * sizeof(double2)));
    BPM_CK(cudaMemcpy(M->node64, node64.data(), n * sizeof(NodeF64), cudaMemcpyHostToDevice));
    BPM_CK(cudaMemcpy(M->mat64, mat64.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    BPM_CK(cudaMalloc(&M->node_pos, np * sizeof(float4)));
    BPM_CK(cudaMalloc(&M->node_mat, np * sizeof(float4)));
    BPM_CK(cudaMalloc(&M->sell_off, off.size() * sizeof(int)));
    BPM_CK(cudaMalloc(&M->sell_ent, ent.size() * sizeof(int2)));
    BPM_CK(cudaMalloc(&M->sell_il, ent_il.size() * sizeof(int2)));
    BPM_CK(cudaMemcpy(M->node_pos, pos.data(), np * sizeof(float4), cudaMemcpyHostToDevice));
    BPM_CK(cudaMemcpy(M->node_mat, nm.data(), np * sizeof(float4), cudaMemcpyHostToDevice));
    BPM_CK(cudaMemcpy(M->sell_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    BPM_CK(cudaMemcpy(M->sell_ent, ent.data(), ent.size() * sizeof(int2), cudaMemcpyHostToDevice));
    BPM_CK(cudaMemcpy(M->sell_il, ent_il.data(), ent_il.size() * sizeof(int2), cudaMemcpyHostToDevice));

    M->nb = nb;
    M->nnz = nnz;
    bpm_mesh_info& I = M->info;
    I.n_nodes = n;
    I.n_pad = np;
    I.k_pad = M->k_pad;
    I.n_tets = nt;
    I.n_boundary = nb;
    I.nnz = nnz;
    I.cg_iters_neumann = it1;
    I.cg_iters_dirichlet = it2;
    I.volume_nm3 = Vsum;
    I.exchange_lambda_max_T = lam;
    I.field_bound_T = lam + an_max + kMu0 * ms_max;
    M->an_max = an_max;
    M->ms_max = ms_max;
    I.cg_residual_neumann = res1;
    I.cg_residual_dirichlet = res2;
    return BPM_OK;
}

}  // namespace bpm
