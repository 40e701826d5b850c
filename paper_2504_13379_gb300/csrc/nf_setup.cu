// nf_setup.cu -- stencils (§3.1) and RBF quadrature weights (§3.2 Eq. (3.5), §3.3
// Eq. (3.6)) on the GPU, in FP64.
//
// Stencils: nodes are binned into a uniform grid; each element's centroid searches
// shells of cells of growing Chebyshev radius, keeping the k smallest
// (distance^2, index) pairs, until no unvisited cell can hold a closer node.  All
// distances use explicitly rounded FP64 operations (no contraction) in a fixed order,
// so the selection equals a brute-force FP64 selection bit for bit.
//
// Weights: one block per element.  Local frame (flat: centroid and max stencil
// radius; surface: projection point from three cutting planes, central projection of
// the stencil to the element plane and the Jacobian of the map), the saddle system of
// Eq. (3.4) with r^3 and monomials up to deg, analytic right-hand side, LU with
// partial pivoting in shared memory, element weights; then a deterministic gather
// q_i = sum of the element weights of every stencil entry naming node i, in ascending
// (element, position) order.
#include "nf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace nfi {

constexpr int KNN_KMAX = 128;

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double dsq(double t) { return __dmul_rn(t, t); }

__device__ __forceinline__ void centroid_of(const double *nodes, int dim, const int32_t *tri, double *c) {
    for (int d = 0; d < dim; ++d) {
        double s = __dadd_rn(nodes[(int64_t)tri[0] * dim + d], nodes[(int64_t)tri[1] * dim + d]);
        s = __dadd_rn(s, nodes[(int64_t)tri[2] * dim + d]);
        c[d] = __ddiv_rn(s, 3.0);
    }
}

__device__ __forceinline__ double exact_d2(const double *x, const double *c, int dim) {
    double s = dsq(__dsub_rn(x[0], c[0]));
    s = __dadd_rn(s, dsq(__dsub_rn(x[1], c[1])));
    if (dim == 3) s = __dadd_rn(s, dsq(__dsub_rn(x[2], c[2])));
    return s;
}

// ------------------------------------------------------------------ input validation
// flag <- 1 if any of the cnt indices is outside [0, n)
__global__ void validate_indices_kernel(const int32_t *idx, int64_t cnt, int64_t n, int *flag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt && (idx[t] < 0 || idx[t] >= n)) atomicExch(flag, 1);
}

// ------------------------------------------------------------------ grid build
struct Grid {
    double lo[3];
    double h;
    int G[3];
    int64_t ncell;
};

__global__ void bbox_partial_kernel(const double *nodes, int64_t n, int dim, double *out) {
    __shared__ double smin[3][256], smax[3][256];
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < dim; ++d) {
            const double v = nodes[j * dim + d];
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    for (int d = 0; d < 3; ++d) {
        smin[d][threadIdx.x] = mn[d];
        smax[d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int d = 0; d < 3; ++d) {
                smin[d][threadIdx.x] = fmin(smin[d][threadIdx.x], smin[d][threadIdx.x + st]);
                smax[d][threadIdx.x] = fmax(smax[d][threadIdx.x], smax[d][threadIdx.x + st]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) {
            out[blockIdx.x * 6 + d] = smin[d][0];
            out[blockIdx.x * 6 + 3 + d] = smax[d][0];
        }
}

__device__ __forceinline__ int cell_coord(double v, double lo, double h, int G) {
    int c = (int)floor((v - lo) / h);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

__global__ void cell_count_kernel(const double *nodes, int64_t n, int dim, Grid gr, int32_t *cell_of,
                                  int32_t *counts) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int c[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) c[d] = cell_coord(nodes[j * dim + d], gr.lo[d], gr.h, gr.G[d]);
    const int32_t id = (int32_t)(((int64_t)c[2] * gr.G[1] + c[1]) * gr.G[0] + c[0]);
    cell_of[j] = id;
    atomicAdd(&counts[id], 1);
}

// single-block exclusive scan (ncell up to a few million; sequential chunks per thread)
__global__ void exclusive_scan_kernel(const int32_t *in, int64_t len, int32_t *out) {
    __shared__ int32_t part[1024];
    const int T = blockDim.x;
    const int64_t per = (len + T - 1) / T;
    const int64_t b = threadIdx.x * per, e = min(len, b + per);
    int32_t s = 0;
    for (int64_t i = b; i < e; ++i) s += in[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int t = 0; t < T; ++t) {
            const int32_t v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    int32_t run = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
        const int32_t v = in[i];
        out[i] = run;
        run += v;
    }
    if (threadIdx.x == T - 1) out[len] = run;
}

__global__ void cell_fill_kernel(int64_t n, const int32_t *cell_of, const int32_t *start, int32_t *fill,
                                 int32_t *sorted) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int32_t c = cell_of[j];
    const int32_t pos = start[c] + atomicAdd(&fill[c], 1);
    sorted[pos] = (int32_t)j;
}

// Query point e: the centroid of triangle e (tris given), or centers[e] (centers given).
__global__ void knn_query_kernel(const double *__restrict__ nodes, int64_t n, int dim,
                                 const int32_t *__restrict__ tris, const double *__restrict__ centers, int64_t m,
                                 int k, Grid gr, const int32_t *__restrict__ start, const int32_t *__restrict__ sorted,
                                 int32_t *__restrict__ stencils) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    double c[3] = {0, 0, 0};
    if (centers) {
        for (int d = 0; d < dim; ++d) c[d] = centers[e * dim + d];
    } else {
        centroid_of(nodes, dim, tris + 3 * e, c);
    }
    int cc[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) cc[d] = cell_coord(c[d], gr.lo[d], gr.h, gr.G[d]);
    double bd[KNN_KMAX];
    int32_t bi[KNN_KMAX];
    int cnt = 0;
    const int gmax = max(gr.G[0], max(gr.G[1], gr.G[2]));
    for (int rho = 0; rho <= gmax; ++rho) {
        const int zr = (dim == 3) ? rho : 0;
        for (int dz = -zr; dz <= zr; ++dz) {
            const int z = cc[2] + dz;
            if (z < 0 || z >= gr.G[2]) continue;
            for (int dy = -rho; dy <= rho; ++dy) {
                const int y = cc[1] + dy;
                if (y < 0 || y >= gr.G[1]) continue;
                for (int dx = -rho; dx <= rho; ++dx) {
                    if (max(abs(dx), max(abs(dy), abs(dz))) != rho) continue;  // shell only
                    const int x = cc[0] + dx;
                    if (x < 0 || x >= gr.G[0]) continue;
                    const int64_t id = ((int64_t)z * gr.G[1] + y) * gr.G[0] + x;
                    for (int32_t p = start[id]; p < start[id + 1]; ++p) {
                        const int32_t j = sorted[p];
                        const double d2 = exact_d2(nodes + (int64_t)j * dim, c, dim);
                        if (cnt == k && !(d2 < bd[k - 1] || (d2 == bd[k - 1] && j < bi[k - 1]))) continue;
                        int pos = (cnt < k) ? cnt : k - 1;
                        while (pos > 0 && (d2 < bd[pos - 1] || (d2 == bd[pos - 1] && j < bi[pos - 1]))) {
                            bd[pos] = bd[pos - 1];
                            bi[pos] = bi[pos - 1];
                            --pos;
                        }
                        bd[pos] = d2;
                        bi[pos] = j;
                        if (cnt < k) ++cnt;
                    }
                }
            }
        }
        // every unvisited node is at least rho * h away from the centroid
        if (cnt == k) {
            const double lim = (double)rho * gr.h;
            if (bd[k - 1] < lim * lim * (1.0 - 1e-9)) break;
        }
    }
    for (int r = 0; r < k; ++r) stencils[e * k + r] = bi[r];
}

}  // namespace nfi

using namespace nfi;

// k nearest nodes to each query point: triangle centroids (tris) or given centres (centers).
// The search grid covers the nodes and, with centres, the centres as well, so that its
// shell-by-shell stopping rule holds for query points outside the nodes' bounding box.
static nf_status build_stencils(const double *nodes, int64_t n, int dim, const int32_t *tris, const double *centers,
                                int64_t m, int k, int32_t *stencils, cudaStream_t s) {
    NF_ARG(dim == 2 || dim == 3, "dim must be 2 or 3 (got %d)", dim);
    NF_ARG(n >= 1 && n < ((int64_t)1 << 31), "n out of range");
    NF_ARG(m >= 1 && m < ((int64_t)1 << 31), "m out of range");
    NF_ARG(k >= 1 && k <= KNN_KMAX && k <= n, "k = %d must satisfy 1 <= k <= min(n, %d)", k, KNN_KMAX);
    // bounding box of the nodes (first nb partials) and of the centres (next nbc)
    const int nb = (int)std::min<int64_t>(256, ceil_div(n, 256));
    const int nbc = centers ? (int)std::min<int64_t>(256, ceil_div(m, 256)) : 0;
    double *dbox = nullptr;
    NF_CUDA_TRY(cudaMallocAsync(&dbox, sizeof(double) * 6 * (nb + nbc) + 16, s));
    int *dflag = reinterpret_cast<int *>(dbox + 6 * (nb + nbc));
    NF_CUDA_TRY(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    if (tris) validate_indices_kernel<<<(unsigned)ceil_div(3 * m, 256), 256, 0, s>>>(tris, 3 * m, n, dflag);
    bbox_partial_kernel<<<nb, 256, 0, s>>>(nodes, n, dim, dbox);
    if (centers) bbox_partial_kernel<<<nbc, 256, 0, s>>>(centers, m, dim, dbox + 6 * nb);
    NF_CUDA_TRY(cudaGetLastError());
    std::vector<double> hbox(6 * (nb + nbc));
    int hflag = 0;
    NF_CUDA_TRY(cudaMemcpyAsync(hbox.data(), dbox, sizeof(double) * 6 * (nb + nbc), cudaMemcpyDeviceToHost, s));
    NF_CUDA_TRY(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    NF_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflag) {
        cudaFreeAsync(dbox, s);
        return fail(NF_ERR_ARG, "tris holds a node index outside [0, n)");
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int b = 0; b < nb + nbc; ++b)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], hbox[6 * b + d]);
            hi[d] = std::max(hi[d], hbox[6 * b + 3 + d]);
        }
    for (int d = 0; d < dim; ++d)
        if (!std::isfinite(lo[d]) || !std::isfinite(hi[d])) {
            cudaFreeAsync(dbox, s);
            return fail(NF_ERR_ARG, "non-finite node or centre coordinates");
        }
    Grid gr{};
    double ext = 0.0;
    for (int d = 0; d < dim; ++d) ext = std::max(ext, hi[d] - lo[d]);
    if (!(ext > 0.0)) ext = 1.0;
    const double per = (dim == 3) ? std::cbrt((double)n / 2.0) : std::sqrt((double)n / 4.0);
    gr.h = ext / std::max(1.0, std::floor(per));
    for (int d = 0; d < 3; ++d) {
        gr.lo[d] = (d < dim) ? lo[d] : 0.0;
        gr.G[d] = (d < dim) ? std::max(1, (int)std::ceil((hi[d] - lo[d]) / gr.h) + 1) : 1;
    }
    gr.ncell = (int64_t)gr.G[0] * gr.G[1] * gr.G[2];
    NF_ARG(gr.ncell < ((int64_t)1 << 30), "degenerate node bounding box");
    int32_t *cell_of = nullptr, *counts = nullptr, *start = nullptr, *sorted = nullptr;
    NF_CUDA_TRY(cudaMallocAsync(&cell_of, sizeof(int32_t) * n, s));
    NF_CUDA_TRY(cudaMallocAsync(&counts, sizeof(int32_t) * gr.ncell, s));
    NF_CUDA_TRY(cudaMallocAsync(&start, sizeof(int32_t) * (gr.ncell + 1), s));
    NF_CUDA_TRY(cudaMallocAsync(&sorted, sizeof(int32_t) * n, s));
    NF_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * gr.ncell, s));
    cell_count_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(nodes, n, dim, gr, cell_of, counts);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(counts, gr.ncell, start);
    NF_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * gr.ncell, s));
    cell_fill_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, cell_of, start, counts, sorted);
    knn_query_kernel<<<(unsigned)ceil_div(m, 128), 128, 0, s>>>(nodes, n, dim, tris, centers, m, k, gr, start,
                                                                sorted, stencils);
    NF_CUDA_TRY(cudaGetLastError());
    cudaFreeAsync(cell_of, s);
    cudaFreeAsync(counts, s);
    cudaFreeAsync(start, s);
    cudaFreeAsync(sorted, s);
    cudaFreeAsync(dbox, s);
    return NF_OK;
}

extern "C" nf_status nf_build_stencils(const double *nodes, int64_t n, int dim, const int32_t *tris, int64_t m,
                                       int k, int32_t *stencils, void *stream) {
    clear_error();
    NF_ARG(nodes && tris && stencils, "nodes, tris and stencils must be non-NULL");
    return build_stencils(nodes, n, dim, tris, nullptr, m, k, stencils, as_stream(stream));
}

extern "C" nf_status nf_build_stencils_at(const double *nodes, int64_t n, int dim, const double *centers, int64_t m,
                                          int k, int32_t *stencils, void *stream) {
    clear_error();
    NF_ARG(nodes && centers && stencils, "nodes, centers and stencils must be non-NULL");
    return build_stencils(nodes, n, dim, nullptr, centers, m, k, stencils, as_stream(stream));
}

// ======================================================================= weights
namespace nfi {

constexpr int QW_THREADS = 128;
constexpr int QW_KMAX = 64;
constexpr int QW_DEGMAX = 4;
constexpr int QW_PMAX = (QW_DEGMAX + 1) * (QW_DEGMAX + 2) / 2;
constexpr double QW_PIVOT_TOL = 1e-14;
constexpr double QW_PROJ_COND_MAX = 1e10;

// ---------------------------------------------------------------- adjacency
constexpr unsigned long long EMPTY_KEY = 0xffffffffffffffffull;

__device__ __forceinline__ unsigned long long edge_key(int32_t a, int32_t b) {
    const unsigned lo = (unsigned)min(a, b), hi = (unsigned)max(a, b);
    return ((unsigned long long)lo << 32) | hi;
}
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

__global__ void edge_insert_kernel(const int32_t *tris, int64_t m, unsigned long long *keys, long long *v0,
                                   long long *v1, int64_t cap, int *flag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * m) return;
    const int64_t e = t / 3;
    const int kk = (int)(t % 3);
    const unsigned long long key = edge_key(tris[3 * e + kk], tris[3 * e + (kk + 1) % 3]);
    int64_t h = (int64_t)(mix64(key) & (unsigned long long)(cap - 1));
    for (int64_t probe = 0; probe < cap; ++probe) {
        const unsigned long long prev = atomicCAS(&keys[h], EMPTY_KEY, key);
        if (prev == EMPTY_KEY || prev == key) {
            if (atomicCAS((unsigned long long *)&v0[h], (unsigned long long)-1ll, (unsigned long long)t) !=
                (unsigned long long)-1ll) {
                if (atomicCAS((unsigned long long *)&v1[h], (unsigned long long)-1ll, (unsigned long long)t) !=
                    (unsigned long long)-1ll)
                    atomicExch(flag, 1);  // edge shared by more than two elements
            }
            return;
        }
        h = (h + 1) & (cap - 1);
    }
    atomicExch(flag, 2);
}

__global__ void edge_lookup_kernel(const int32_t *tris, int64_t m, const unsigned long long *keys,
                                   const long long *v0, const long long *v1, int64_t cap, const int *flag,
                                   int64_t *nbr) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * m) return;
    const int64_t e = t / 3;
    const int kk = (int)(t % 3);
    const unsigned long long key = edge_key(tris[3 * e + kk], tris[3 * e + (kk + 1) % 3]);
    int64_t h = (int64_t)(mix64(key) & (unsigned long long)(cap - 1));
    nbr[t] = -1;
    if (*flag) return;  // non-manifold: every element falls back to parallel projection
    for (int64_t probe = 0; probe < cap; ++probe) {
        if (keys[h] == key) {
            const long long a = v0[h], b = v1[h];
            const long long other = (a == t) ? b : a;
            nbr[t] = (other >= 0) ? other / 3 : -1;
            return;
        }
        if (keys[h] == EMPTY_KEY) return;
        h = (h + 1) & (cap - 1);
    }
}

// ---------------------------------------------------------------- small geometry
struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 v3(const double *p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 scl(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double nrm(V3 a) { return sqrt(dot(a, a)); }

__device__ V3 element_normal(const double *X, const double *NS, const int32_t *tri) {
    const V3 a = v3(X + 3 * (int64_t)tri[0]), b = v3(X + 3 * (int64_t)tri[1]), c = v3(X + 3 * (int64_t)tri[2]);
    V3 nE = cross(sub(b, a), sub(c, a));
    nE = scl(nE, 1.0 / nrm(nE));
    const V3 ref = add(add(v3(NS + 3 * (int64_t)tri[0]), v3(NS + 3 * (int64_t)tri[1])), v3(NS + 3 * (int64_t)tri[2]));
    if (dot(nE, ref) < 0.0) nE = scl(nE, -1.0);
    return nE;
}

// Solve A p = b (3x3) via the Gauss-Jordan inverse; returns ||A||_inf ||A^-1||_inf.
__device__ double solve3x3(const double A[9], const double b[3], double p[3]) {
    double W[3][6];
    double anorm = 0.0;
    for (int r = 0; r < 3; ++r) {
        anorm = fmax(anorm, fabs(A[3 * r]) + fabs(A[3 * r + 1]) + fabs(A[3 * r + 2]));
        for (int c = 0; c < 6; ++c) W[r][c] = (c < 3) ? A[3 * r + c] : (c - 3 == r ? 1.0 : 0.0);
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(W[r][c]) > fabs(W[piv][c])) piv = r;
        if (W[piv][c] == 0.0) return INFINITY;
        if (piv != c)
            for (int cc = 0; cc < 6; ++cc) {
                const double t = W[c][cc];
                W[c][cc] = W[piv][cc];
                W[piv][cc] = t;
            }
        const double pv = W[c][c];
        for (int cc = 0; cc < 6; ++cc) W[c][cc] /= pv;
        for (int r = 0; r < 3; ++r) {
            if (r == c) continue;
            const double l = W[r][c];
            for (int cc = 0; cc < 6; ++cc) W[r][cc] -= l * W[c][cc];
        }
    }
    double inorm = 0.0;
    for (int r = 0; r < 3; ++r) inorm = fmax(inorm, fabs(W[r][3]) + fabs(W[r][4]) + fabs(W[r][5]));
    for (int r = 0; r < 3; ++r) p[r] = W[r][3] * b[0] + W[r][4] * b[1] + W[r][5] * b[2];
    return anorm * inorm;
}

// ---------------------------------------------------------------- analytic integrals
// d^5 G(a/d), G the antiderivative of sec^5 (polar integral of r^3 over a fan wedge).
__device__ __forceinline__ double sec5_wedge(double a, double d) {
    const double rr = sqrt(a * a + d * d);
    const double d2 = d * d;
    return 0.25 * d * a * rr * rr * rr + 0.375 * d2 * d * a * rr + 0.375 * d2 * d2 * d * asinh(a / d);
}

// int_T |x - p|^3 dx, T given by 3 vertices (x0,y0,x1,y1,x2,y2), any orientation.
__device__ double tri_r3_integral(double px, double py, const double *v) {
    const double area2 = (v[2] - v[0]) * (v[5] - v[1]) - (v[3] - v[1]) * (v[4] - v[0]);
    double total = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double Ax = v[2 * e], Ay = v[2 * e + 1];
        const double Bx = v[2 * ((e + 1) % 3)], By = v[2 * ((e + 1) % 3) + 1];
        const double ex = Bx - Ax, ey = By - Ay;
        const double L = sqrt(ex * ex + ey * ey);
        const double tx = ex / L, ty = ey / L;
        const double ax = Ax - px, ay = Ay - py;
        const double cr = ax * ty - ay * tx;
        const double d = fabs(cr);
        if (d == 0.0) continue;
        const double aA = ax * tx + ay * ty;
        const double part = (sec5_wedge(aA + L, d) - sec5_wedge(aA, d)) / 5.0;
        total += (cr > 0.0) ? part : -part;
    }
    return area2 > 0.0 ? total : -total;
}

__device__ __forceinline__ double ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}
__device__ __forceinline__ double fact(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

// int_T x^a y^b: barycentric expansion, int_T l0^i l1^j l2^k = 2|T| i! j! k! / (i+j+k+2)!
__device__ double tri_monomial_integral(int a, int b, const double *v) {
    const double area = 0.5 * fabs((v[2] - v[0]) * (v[5] - v[1]) - (v[3] - v[1]) * (v[4] - v[0]));
    double total = 0.0;
    for (int i0 = 0; i0 <= a; ++i0)
        for (int i1 = 0; i0 + i1 <= a; ++i1) {
            const int i2 = a - i0 - i1;
            const double cx = fact(a) / (fact(i0) * fact(i1) * fact(i2)) * ipow(v[0], i0) * ipow(v[2], i1) *
                              ipow(v[4], i2);
            for (int j0 = 0; j0 <= b; ++j0)
                for (int j1 = 0; j0 + j1 <= b; ++j1) {
                    const int j2 = b - j0 - j1;
                    const double cy = fact(b) / (fact(j0) * fact(j1) * fact(j2)) * ipow(v[1], j0) *
                                      ipow(v[3], j1) * ipow(v[5], j2);
                    total += cx * cy * 2.0 * area * fact(i0 + j0) * fact(i1 + j1) * fact(i2 + j2) / fact(a + b + 2);
                }
        }
    return total;
}

// ---------------------------------------------------------------- per-element solve
struct QwArgs {
    const double *X;
    const double *NS;   // null when flat
    int dim;
    const int32_t *tris;
    int64_t m;
    const int32_t *sten;
    int k;
    int deg;
    const int64_t *nbr;  // 3 per element (surfaces)
    double *elem_w;      // m x k
    unsigned long long *first_bad;
};

__global__ void __launch_bounds__(QW_THREADS) quad_element_kernel(QwArgs a) {
    extern __shared__ __align__(16) double qsm[];
    const int k = a.k;
    const int P = (a.deg + 1) * (a.deg + 2) / 2;
    const int N = k + P;
    const int ld = N + 1;
    double *M = qsm;                  // N x ld
    double *z = M + (size_t)N * ld;   // N
    double *xi = z + N;               // 2k local coordinates
    double *jac = xi + 2 * k;         // k
    double *tv = jac + k;             // 6 triangle vertices
    double *misc = tv + 6;            // frame: [0..2] c, [3..5] e1, [6..8] e2, [9..11] nE, [12..14] p, [15] central, [16] rho, [17] anorm, [18] best, [19] piv
    __shared__ int s_ea[QW_PMAX], s_eb[QW_PMAX];
    const int tid = threadIdx.x;
    const int64_t e = blockIdx.x;
    const int32_t *S = a.sten + e * k;
    const int32_t *tri = a.tris + 3 * e;

    if (tid == 0) {
        int c = 0;
        for (int t = 0; t <= a.deg; ++t)
            for (int ax = t; ax >= 0; --ax) {
                s_ea[c] = ax;
                s_eb[c] = t - ax;
                ++c;
            }
        if (a.dim == 2) {
            for (int d = 0; d < 2; ++d)
                misc[d] = ((a.X[2 * (int64_t)tri[0] + d] + a.X[2 * (int64_t)tri[1] + d]) + a.X[2 * (int64_t)tri[2] + d]) /
                          3.0;
        } else {
            const V3 A = v3(a.X + 3 * (int64_t)tri[0]), B = v3(a.X + 3 * (int64_t)tri[1]), Cc = v3(a.X + 3 * (int64_t)tri[2]);
            const V3 cE = {((A.x + B.x) + Cc.x) / 3.0, ((A.y + B.y) + Cc.y) / 3.0, ((A.z + B.z) + Cc.z) / 3.0};
            const V3 nE = element_normal(a.X, a.NS, tri);
            V3 e1 = sub(B, A);
            e1 = scl(e1, 1.0 / nrm(e1));
            const V3 e2 = cross(nE, e1);
            double Am[9], rhs[3], p[3] = {0, 0, 0};
            bool central = true;
            for (int kk = 0; kk < 3; ++kk) {
                const int64_t f = a.nbr[3 * e + kk];
                if (f < 0) {
                    central = false;
                    break;
                }
                const V3 nF = element_normal(a.X, a.NS, a.tris + 3 * f);
                const V3 dn = sub(nE, nF);
                Am[3 * kk] = dn.x;
                Am[3 * kk + 1] = dn.y;
                Am[3 * kk + 2] = dn.z;
                rhs[kk] = dot(dn, v3(a.X + 3 * (int64_t)tri[kk]));
            }
            if (central) {
                const double cond = solve3x3(Am, rhs, p);
                central = isfinite(cond) && cond < QW_PROJ_COND_MAX;
            }
            misc[0] = cE.x; misc[1] = cE.y; misc[2] = cE.z;
            misc[3] = e1.x; misc[4] = e1.y; misc[5] = e1.z;
            misc[6] = e2.x; misc[7] = e2.y; misc[8] = e2.z;
            misc[9] = nE.x; misc[10] = nE.y; misc[11] = nE.z;
            misc[12] = p[0]; misc[13] = p[1]; misc[14] = p[2];
            misc[15] = central ? 1.0 : 0.0;
        }
    }
    __syncthreads();

    // project stencil nodes to the element plane (surfaces) and measure rho
    // xi temporarily holds in-plane offsets (3D -> stored 2D after the frame is known)
    for (int r = tid; r < k; r += blockDim.x) {
        const int64_t j = S[r];
        if (a.dim == 2) {
            xi[2 * r] = a.X[2 * j] - misc[0];
            xi[2 * r + 1] = a.X[2 * j + 1] - misc[1];
            jac[r] = 1.0;
        } else {
            const V3 x = v3(a.X + 3 * j), ns = v3(a.NS + 3 * j);
            const V3 cE = {misc[0], misc[1], misc[2]}, e1 = {misc[3], misc[4], misc[5]}, e2 = {misc[6], misc[7], misc[8]};
            const V3 nE = {misc[9], misc[10], misc[11]}, p = {misc[12], misc[13], misc[14]};
            V3 xp3;
            if (misc[15] != 0.0) {
                const V3 xp = sub(x, p);
                const double t = dot(sub(cE, p), nE) / dot(xp, nE);
                const double lx = nrm(xp);
                const V3 u = scl(xp, 1.0 / lx);
                xp3 = add(p, scl(xp, t));
                jac[r] = (1.0 / (t * t)) * fabs(dot(nE, u)) / fabs(dot(ns, u));
            } else {
                const double sd = dot(sub(x, cE), nE);
                xp3 = sub(x, scl(nE, sd));
                jac[r] = 1.0 / fabs(dot(ns, nE));
            }
            const V3 v = sub(xp3, cE);
            xi[2 * r] = dot(v, e1);
            xi[2 * r + 1] = dot(v, e2);
        }
    }
    __syncthreads();
    if (tid == 0) {
        double rho = 0.0;
        for (int r = 0; r < k; ++r) rho = fmax(rho, sqrt(xi[2 * r] * xi[2 * r] + xi[2 * r + 1] * xi[2 * r + 1]));
        misc[16] = rho;
        for (int i = 0; i < 3; ++i) {
            const int64_t j = tri[i];
            if (a.dim == 2) {
                tv[2 * i] = (a.X[2 * j] - misc[0]) / rho;
                tv[2 * i + 1] = (a.X[2 * j + 1] - misc[1]) / rho;
            } else {
                const V3 v = sub(v3(a.X + 3 * j), V3{misc[0], misc[1], misc[2]});
                tv[2 * i] = dot(v, V3{misc[3], misc[4], misc[5]}) / rho;
                tv[2 * i + 1] = dot(v, V3{misc[6], misc[7], misc[8]}) / rho;
            }
        }
    }
    __syncthreads();
    const double rho = misc[16];
    for (int r = tid; r < k; r += blockDim.x) {
        xi[2 * r] /= rho;
        xi[2 * r + 1] /= rho;
    }
    __syncthreads();

    // assemble the saddle system of Eq. (3.4) and its right-hand side; the matrix is
    // symmetric, so each entry of the upper triangle is computed once and mirrored (the
    // kernel is bound by the FP64 pipe, and the r^3 entries' square roots dominate the
    // assembly)
    for (int idx = tid; idx < N * N; idx += blockDim.x) {
        const int r = idx / N, c = idx % N;
        if (c < r) continue;
        double v;
        if (r < k && c < k) {
            const double dx = xi[2 * r] - xi[2 * c], dy = xi[2 * r + 1] - xi[2 * c + 1];
            const double rr = sqrt(dx * dx + dy * dy);
            v = rr * rr * rr;
        } else if (r < k) {
            v = ipow(xi[2 * r], s_ea[c - k]) * ipow(xi[2 * r + 1], s_eb[c - k]);
        } else if (c < k) {
            v = ipow(xi[2 * c], s_ea[r - k]) * ipow(xi[2 * c + 1], s_eb[r - k]);
        } else {
            v = 0.0;
        }
        M[r * ld + c] = v;
        M[c * ld + r] = v;
    }
    for (int r = tid; r < N; r += blockDim.x)
        z[r] = (r < k) ? tri_r3_integral(xi[2 * r], xi[2 * r + 1], tv)
                       : tri_monomial_integral(s_ea[r - k], s_eb[r - k], tv);
    __syncthreads();
    if (tid < 32) {
        double mx = 0.0;
        for (int r = tid; r < N; r += 32) {
            double sacc = 0.0;
            for (int c = 0; c < N; ++c) sacc += fabs(M[r * ld + c]);
            mx = fmax(mx, sacc);
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (tid == 0) misc[17] = mx;
    }
    __syncthreads();
    const double anorm = misc[17];

    // LU with partial pivoting (first maximal pivot); each elimination update is one fused
    // multiply-add (the FP64 pipe bounds this kernel, and the fusion halves its updates)
    for (int c = 0; c < N; ++c) {
        if (tid < 32) {
            double best = -1.0;
            int piv = N;
            for (int r = c + tid; r < N; r += 32) {
                const double v = fabs(M[r * ld + c]);
                if (v > best) {
                    best = v;
                    piv = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int op = __shfl_xor_sync(0xffffffffu, piv, o);
                if (ob > best || (ob == best && op < piv)) {
                    best = ob;
                    piv = op;
                }
            }
            if (tid == 0) {
                misc[18] = best;
                misc[19] = (double)piv;
            }
        }
        __syncthreads();
        const double best = misc[18];
        const int piv = (int)misc[19];
        if (!(best > QW_PIVOT_TOL * anorm)) {
            if (tid == 0) atomicMin(a.first_bad, (unsigned long long)e);
            return;  // uniform across the block
        }
        if (piv != c) {
            for (int cc = tid; cc < N; cc += blockDim.x) {
                const double t = M[c * ld + cc];
                M[c * ld + cc] = M[piv * ld + cc];
                M[piv * ld + cc] = t;
            }
            if (tid == 0) {
                const double t = z[c];
                z[c] = z[piv];
                z[piv] = t;
            }
        }
        __syncthreads();
        const double diag = M[c * ld + c];
        for (int r = c + 1 + tid; r < N; r += blockDim.x) M[r * ld + c] = __ddiv_rn(M[r * ld + c], diag);
        __syncthreads();
        const int rows = N - c - 1;
        const int cols = N - c;  // columns c+1..N-1 plus the right-hand side
        for (int idx = tid; idx < rows * cols; idx += blockDim.x) {
            const int r = c + 1 + idx / cols;
            const int cc = c + 1 + idx % cols;
            const double l = M[r * ld + c];
            if (cc < N)
                M[r * ld + cc] = __fma_rn(-l, M[c * ld + cc], M[r * ld + cc]);
            else
                z[r] = __fma_rn(-l, z[c], z[r]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        for (int r = N - 1; r >= 0; --r) {
            double sacc = z[r];
            for (int cc = r + 1; cc < N; ++cc) sacc = __fma_rn(-M[r * ld + cc], z[cc], sacc);
            z[r] = __ddiv_rn(sacc, M[r * ld + r]);
        }
    }
    __syncthreads();
    for (int r = tid; r < k; r += blockDim.x) a.elem_w[e * k + r] = z[r] * rho * rho * jac[r];
}

// ---------------------------------------------------------------- deterministic gather
__global__ void count_refs_kernel(const int32_t *sten, int64_t mk, int32_t *cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < mk) atomicAdd(&cnt[sten[t]], 1);
}
__global__ void fill_refs_kernel(const int32_t *sten, int64_t mk, const int32_t *start, int32_t *fill,
                                 int64_t *refs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mk) return;
    const int32_t i = sten[t];
    refs[start[i] + atomicAdd(&fill[i], 1)] = t;
}
// q_i = sum over its references in ascending flat (element * k + position) order
__global__ void gather_weights_kernel(int64_t n, const int32_t *start, int64_t *refs, const double *elem_w,
                                      double *q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t b = start[i], e = start[i + 1];
    for (int32_t p = b + 1; p < e; ++p) {  // insertion sort of this node's references
        const int64_t v = refs[p];
        int32_t s = p;
        while (s > b && refs[s - 1] > v) {
            refs[s] = refs[s - 1];
            --s;
        }
        refs[s] = v;
    }
    double acc = 0.0;
    for (int32_t p = b; p < e; ++p) acc += elem_w[refs[p]];
    q[i] = acc;
}

}  // namespace nfi

extern "C" nf_status nf_quad_weights(const double *nodes, const double *normals, int64_t n, int dim,
                                     const int32_t *tris, int64_t m, const int32_t *stencils, int k, int deg,
                                     double *q, int64_t *bad_element, void *stream) {
    clear_error();
    if (bad_element) *bad_element = -1;
    NF_ARG(nodes && tris && stencils && q, "nodes, tris, stencils and q must be non-NULL");
    NF_ARG(dim == 2 || dim == 3, "dim must be 2 or 3");
    NF_ARG((dim == 3) == (normals != nullptr), "normals are required for dim 3 and must be NULL for dim 2");
    NF_ARG(n >= 3 && n < ((int64_t)1 << 31) && m >= 1 && m < ((int64_t)1 << 31), "n or m out of range");
    NF_ARG(deg >= 0 && deg <= QW_DEGMAX, "deg must be in 0..%d", QW_DEGMAX);
    const int P = (deg + 1) * (deg + 2) / 2;
    NF_ARG(k >= P, "k = %d is below the %d polynomial terms of degree %d (unisolvency)", k, P, deg);
    NF_ARG(k <= QW_KMAX && k <= n, "k = %d must be <= min(n, %d)", k, QW_KMAX);
    cudaStream_t s = as_stream(stream);
    const int N = k + P;
    const size_t smem = sizeof(double) * ((size_t)N * (N + 1) + N + 3 * (size_t)k + 6 + 24);
    // per call: the attribute belongs to the current device, and a call costs microseconds
    NF_CUDA_TRY(cudaFuncSetAttribute(quad_element_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t *nbr = nullptr;
    unsigned long long *keys = nullptr;
    long long *v0 = nullptr, *v1 = nullptr;
    int *flag = nullptr;
    unsigned long long *first_bad = nullptr;
    double *elem_w = nullptr;
    NF_CUDA_TRY(cudaMallocAsync(&first_bad, 64, s));
    flag = reinterpret_cast<int *>(reinterpret_cast<char *>(first_bad) + 16);
    NF_CUDA_TRY(cudaMemsetAsync(first_bad, 0xff, 8, s));
    NF_CUDA_TRY(cudaMemsetAsync(flag, 0, 4, s));
    {
        validate_indices_kernel<<<(unsigned)ceil_div(3 * m, 256), 256, 0, s>>>(tris, 3 * m, n, flag);
        validate_indices_kernel<<<(unsigned)ceil_div(m * k, 256), 256, 0, s>>>(stencils, m * k, n, flag);
        int hflag = 0;
        NF_CUDA_TRY(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        NF_CUDA_TRY(cudaStreamSynchronize(s));
        if (hflag) {
            cudaFreeAsync(first_bad, s);
            return fail(NF_ERR_ARG, "tris or stencils hold a node index outside [0, n)");
        }
    }
    NF_CUDA_TRY(cudaMallocAsync(&elem_w, sizeof(double) * m * k, s));
    if (dim == 3) {
        int64_t cap = 1;
        while (cap < 4 * 3 * m) cap <<= 1;
        NF_CUDA_TRY(cudaMallocAsync(&nbr, sizeof(int64_t) * 3 * m, s));
        NF_CUDA_TRY(cudaMallocAsync(&keys, sizeof(unsigned long long) * cap, s));
        NF_CUDA_TRY(cudaMallocAsync(&v0, sizeof(long long) * cap, s));
        NF_CUDA_TRY(cudaMallocAsync(&v1, sizeof(long long) * cap, s));
        NF_CUDA_TRY(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * cap, s));
        NF_CUDA_TRY(cudaMemsetAsync(v0, 0xff, sizeof(long long) * cap, s));
        NF_CUDA_TRY(cudaMemsetAsync(v1, 0xff, sizeof(long long) * cap, s));
        edge_insert_kernel<<<(unsigned)ceil_div(3 * m, 256), 256, 0, s>>>(tris, m, keys, v0, v1, cap, flag);
        edge_lookup_kernel<<<(unsigned)ceil_div(3 * m, 256), 256, 0, s>>>(tris, m, keys, v0, v1, cap, flag, nbr);
        NF_CUDA_TRY(cudaGetLastError());
    }
    QwArgs qa{nodes, normals, dim, tris, m, stencils, k, deg, nbr, elem_w, first_bad};
    quad_element_kernel<<<(unsigned)m, QW_THREADS, smem, s>>>(qa);
    NF_CUDA_TRY(cudaGetLastError());
    int32_t *cnt = nullptr, *start = nullptr;
    int64_t *refs = nullptr;
    NF_CUDA_TRY(cudaMallocAsync(&cnt, sizeof(int32_t) * n, s));
    NF_CUDA_TRY(cudaMallocAsync(&start, sizeof(int32_t) * (n + 1), s));
    NF_CUDA_TRY(cudaMallocAsync(&refs, sizeof(int64_t) * m * k, s));
    NF_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s));
    count_refs_kernel<<<(unsigned)ceil_div(m * k, 256), 256, 0, s>>>(stencils, m * k, cnt);
    exclusive_scan_kernel<<<1, 1024, 0, s>>>(cnt, n, start);
    NF_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s));
    fill_refs_kernel<<<(unsigned)ceil_div(m * k, 256), 256, 0, s>>>(stencils, m * k, start, cnt, refs);
    gather_weights_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, start, refs, elem_w, q);
    NF_CUDA_TRY(cudaGetLastError());
    unsigned long long hbad = ~0ull;
    NF_CUDA_TRY(cudaMemcpyAsync(&hbad, first_bad, 8, cudaMemcpyDeviceToHost, s));
    NF_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFreeAsync(cnt, s);
    cudaFreeAsync(start, s);
    cudaFreeAsync(refs, s);
    cudaFreeAsync(elem_w, s);
    cudaFreeAsync(first_bad, s);
    if (nbr) cudaFreeAsync(nbr, s);
    if (keys) cudaFreeAsync(keys, s);
    if (v0) cudaFreeAsync(v0, s);
    if (v1) cudaFreeAsync(v1, s);
    NF_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad != ~0ull) {
        if (bad_element) *bad_element = (int64_t)hbad;
        return fail(NF_ERR_SINGULAR, "singular interpolation system at element %lld", (long long)hbad);
    }
    return NF_OK;
}

extern "C" nf_status nf_quad_weights_opts(const double *nodes, const double *normals, int64_t n, const int32_t *tris,
                                          int64_t m, const int32_t *stencils, int k, const nf_quad_opts *o, double *q,
                                          int64_t *bad_element, void *stream) {
    clear_error();
    NF_ARG(o, "options must be non-NULL");
    NF_ARG(o->dim == 2 || o->dim == 3, "dim must be 2 or 3 (got %d)", o->dim);
    NF_ARG(o->curved == (o->dim == 3 ? 1 : 0), "curved must be 1 for dim 3 (surfaces) and 0 for dim 2");
    if (o->phs_order != 3)
        return fail(NF_ERR_UNSUPPORTED, "phs_order %d: the polyharmonic spline r^3 is implemented", o->phs_order);
    return nf_quad_weights(nodes, o->curved ? normals : nullptr, n, o->dim, tris, m, stencils, k, o->poly_deg, q,
                           bad_element, stream);
}
