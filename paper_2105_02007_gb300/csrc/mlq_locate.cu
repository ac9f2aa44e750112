// mlq_locate.cu -- P1 values at arbitrary points by point location on the
// device: the intergrid transfer between meshes that are not nested (Sec. 4,
// Sec. 5.4), e.g. the finest-mesh KL modes at the element centroids of an
// unrelated coarser mesh.
//
// The rule is that of the host helper mlq_p1_at_points: a point takes the
// first simplex, in element order, whose barycentric coordinates are all
// >= -1e-12; a point in no simplex takes the first simplex whose smallest
// coordinate is within 1e-12 of the largest smallest coordinate over all
// simplices, and the linear extension of its P1 function.  Barycentric
// coordinates are ratios of signed measures (x replacing one vertex at a
// time).  Steps, all on the device:
//   1. a uniform grid of buckets over the node bounding box (g per axis,
//      g = round((ne / 6)^(1/dim)) clamped to 1..512); each simplex is listed
//      in every bucket its bounding box meets (count, scan, fill);
//   2. one thread per point scans its bucket's list and keeps the smallest
//      element index whose coordinates pass (the lists are filled in any
//      order, so the minimum stands for "first in element order");
//   3. the points found in no simplex: one CTA each scans every simplex
//      (block maximum of the smallest coordinate, then the smallest index
//      within 1e-12 of it);
//   4. the P1 values of the K fields.
#include "mlq.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace {

constexpr int kT = 256;
constexpr int kScan = 1024;   // entries per CTA of the bucket-count scan

struct LocMesh {
    int d;
    int64_t n, ne;
    const double *xyz;
    const int32_t *conn;
};

struct Grid {
    int g, dim;
    double lo[3], inv[3];
};

__device__ __forceinline__ int grid_cell(const Grid &G, int c, double v)
{
    const int i = (int)floor((v - G.lo[c]) * G.inv[c]);
    return i < 0 ? 0 : (i >= G.g ? G.g - 1 : i);
}

// barycentric coordinates of x in simplex e (ratios of signed measures);
// returns the smallest
__device__ double simplex_bary(const LocMesh &m, int64_t e, const double *x, double *lam)
{
    const int nv = m.d + 1;
    double P[4][3];
    for (int a = 0; a < nv; ++a)
        for (int c = 0; c < 3; ++c) P[a][c] = c < m.d ? m.xyz[(int64_t)m.conn[e * nv + a] * m.d + c] : 0.0;
    auto measure = [&](int skip) {
        // signed measure with vertex `skip` replaced by x (skip = -1: none)
        double Q[4][3];
        for (int a = 0; a < nv; ++a)
            for (int c = 0; c < 3; ++c) Q[a][c] = (a == skip && c < m.d) ? x[c] : P[a][c];
        if (m.d == 2) return (Q[1][0] - Q[0][0]) * (Q[2][1] - Q[0][1]) - (Q[1][1] - Q[0][1]) * (Q[2][0] - Q[0][0]);
        const double u[3] = {Q[1][0] - Q[0][0], Q[1][1] - Q[0][1], Q[1][2] - Q[0][2]};
        const double v[3] = {Q[2][0] - Q[0][0], Q[2][1] - Q[0][1], Q[2][2] - Q[0][2]};
        const double w[3] = {Q[3][0] - Q[0][0], Q[3][1] - Q[0][1], Q[3][2] - Q[0][2]};
        return u[0] * (v[1] * w[2] - v[2] * w[1]) + u[1] * (v[2] * w[0] - v[0] * w[2]) +
               u[2] * (v[0] * w[1] - v[1] * w[0]);
    };
    const double whole = measure(-1);
    double mn = 1e300;
    for (int a = 0; a < nv; ++a) {
        lam[a] = measure(a) / whole;
        mn = fmin(mn, lam[a]);
    }
    return mn;
}

// bucket range of simplex e's bounding box, r[2c], r[2c+1] per axis
__device__ void simplex_box(const LocMesh &m, const Grid &G, int64_t e, int (&r)[6])
{
    const int nv = m.d + 1;
    for (int c = 0; c < 3; ++c) {
        r[2 * c] = 0;
        r[2 * c + 1] = 0;
    }
    for (int c = 0; c < m.d; ++c) {
        double a = 1e300, b = -1e300;
        for (int q = 0; q < nv; ++q) {
            const double v = m.xyz[(int64_t)m.conn[e * nv + q] * m.d + c];
            a = fmin(a, v);
            b = fmax(b, v);
        }
        r[2 * c] = grid_cell(G, c, a);
        r[2 * c + 1] = grid_cell(G, c, b);
    }
}

__global__ void box_count_kernel(LocMesh m, Grid G, unsigned long long *cnt)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    int r[6];
    simplex_box(m, G, e, r);
    for (int z = r[4]; z <= r[5]; ++z)
        for (int y = r[2]; y <= r[3]; ++y)
            for (int x = r[0]; x <= r[1]; ++x) atomicAdd(cnt + (x + (int64_t)G.g * (y + (int64_t)G.g * z)), 1ull);
}

// exclusive scan of cnt[0..nb) into start[0..nb], in CTAs of kScan entries:
// each CTA scans its entries and leaves its total in part[]; part is then
// scanned by one CTA, and each CTA adds its offset
__global__ void scan_local_kernel(int64_t nb, const unsigned long long *cnt, unsigned long long *start,
                                  unsigned long long *part)
{
    __shared__ unsigned long long sh[kScan];
    const int64_t base = (int64_t)blockIdx.x * kScan;
    for (int t = threadIdx.x; t < kScan; t += blockDim.x) sh[t] = base + t < nb ? cnt[base + t] : 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int t = 0; t < kScan; ++t) {
            const unsigned long long v = sh[t];
            sh[t] = acc;
            acc += v;
        }
        part[blockIdx.x] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kScan; t += blockDim.x)
        if (base + t < nb) start[base + t] = sh[t];
}

__global__ void scan_parts_kernel(int64_t nparts, unsigned long long *part, int64_t nb, unsigned long long *start)
{
    if (threadIdx.x != 0) return;
    unsigned long long acc = 0;
    for (int64_t k = 0; k < nparts; ++k) {
        const unsigned long long v = part[k];
        part[k] = acc;
        acc += v;
    }
    start[nb] = acc;
}

__global__ void scan_add_kernel(int64_t nb, const unsigned long long *part, unsigned long long *start,
                                unsigned long long *fill)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const unsigned long long s = start[b] + part[b / kScan];
    start[b] = s;
    fill[b] = s;
}

__global__ void box_fill_kernel(LocMesh m, Grid G, unsigned long long *fill, int32_t *list)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.ne) return;
    int r[6];
    simplex_box(m, G, e, r);
    for (int z = r[4]; z <= r[5]; ++z)
        for (int y = r[2]; y <= r[3]; ++y)
            for (int x = r[0]; x <= r[1]; ++x)
                list[atomicAdd(fill + (x + (int64_t)G.g * (y + (int64_t)G.g * z)), 1ull)] = (int32_t)e;
}

// one thread per point: the smallest element index among the simplices of
// its bucket that contain it (-1: none)
__global__ void locate_kernel(LocMesh m, Grid G, const unsigned long long *start, const int32_t *list, int64_t np,
                              const double *pts, int32_t *elem, double *lam_out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double x[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < m.d; ++c) x[c] = pts[p * m.d + c];
    int64_t b = 0, stride = 1;
    for (int c = 0; c < m.d; ++c) {
        b += grid_cell(G, c, x[c]) * stride;
        stride *= G.g;
    }
    int32_t best = -1;
    double lam[4] = {0.0, 0.0, 0.0, 0.0}, best_lam[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned long long t = start[b]; t < start[b + 1]; ++t) {
        const int32_t e = list[t];
        if (best >= 0 && e >= best) continue;
        if (simplex_bary(m, e, x, lam) >= -1e-12) {
            best = e;
            for (int a = 0; a < 4; ++a) best_lam[a] = lam[a];
        }
    }
    elem[p] = best;
    for (int a = 0; a < 4; ++a) lam_out[p * 4 + a] = best_lam[a];
}

// one CTA per point found in no simplex: the first simplex whose smallest
// coordinate is within 1e-12 of the largest over all simplices
__global__ void outside_kernel(LocMesh m, const double *pts, const int64_t *which, int32_t *elem, double *lam_out)
{
    __shared__ double smax[kT];
    __shared__ long long smin[kT];
    const int64_t p = which[blockIdx.x];
    double x[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < m.d; ++c) x[c] = pts[p * m.d + c];
    double lam[4] = {0.0, 0.0, 0.0, 0.0};
    double mx = -1e300;
    for (int64_t e = threadIdx.x; e < m.ne; e += blockDim.x) mx = fmax(mx, simplex_bary(m, e, x, lam));
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        __syncthreads();
    }
    const double best_min = smax[0];
    long long first = m.ne;
    for (int64_t e = threadIdx.x; e < m.ne && e < first; e += blockDim.x)
        if (simplex_bary(m, e, x, lam) >= best_min - 1e-12) first = e;
    smin[threadIdx.x] = first;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) smin[threadIdx.x] = min(smin[threadIdx.x], smin[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t e = smin[0];
        simplex_bary(m, e, x, lam);
        elem[p] = (int32_t)e;
        for (int a = 0; a < 4; ++a) lam_out[p * 4 + a] = a <= m.d ? lam[a] : 0.0;
    }
}

__global__ void interp_kernel(LocMesh m, int K, const double *f, int64_t np, const int32_t *elem,
                              const double *lam, double *out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np * K) return;
    const int64_t p = t / K;
    const int k = (int)(t - p * K);
    const int nv = m.d + 1;
    const int64_t e = elem[p];
    double v = 0.0;
    for (int a = 0; a < nv; ++a) v += lam[p * 4 + a] * f[(int64_t)m.conn[e * nv + a] * K + k];
    out[t] = v;
}

}  // namespace

extern "C" int mlq_p1_at_points_gpu(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int K,
                                    const double *f, int64_t np, const double *pts, double *out)
{
    if ((dim != 2 && dim != 3) || n < dim + 1 || ne < 1 || ne > INT32_MAX || !xyz || !conn || K < 1 || np < 0)
        return MLQ_EINVAL;
    if (np > 0 && (!f || !pts || !out)) return MLQ_EINVAL;
    const int nv = dim + 1;
    for (int64_t t = 0; t < ne * nv; ++t)
        if (conn[t] < 0 || conn[t] >= n) return MLQ_EINVAL;
    if (np == 0) return MLQ_OK;
    Grid G{};
    G.dim = dim;
    G.g = std::max(1, std::min(512, (int)std::lround(std::pow((double)ne / 6.0, 1.0 / dim))));
    double hi[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < dim; ++c) G.lo[c] = hi[c] = xyz[c];
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < dim; ++c) {
            G.lo[c] = std::min(G.lo[c], xyz[i * dim + c]);
            hi[c] = std::max(hi[c], xyz[i * dim + c]);
        }
    for (int c = 0; c < 3; ++c) G.inv[c] = (c < dim && hi[c] > G.lo[c]) ? G.g / (hi[c] - G.lo[c]) : 1.0;
    int64_t nb = 1;
    for (int c = 0; c < dim; ++c) nb *= G.g;
    const int64_t nparts = (nb + kScan - 1) / kScan;
    std::vector<void *> allocs;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 8)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        allocs.push_back(p);
        return p;
    };
    auto release = [&]() {
        for (void *p : allocs) cudaFree(p);
    };
    double *d_xyz = (double *)alloc(sizeof(double) * n * dim), *d_f = (double *)alloc(sizeof(double) * n * K);
    double *d_pts = (double *)alloc(sizeof(double) * np * dim), *d_out = (double *)alloc(sizeof(double) * np * K);
    double *d_lam = (double *)alloc(sizeof(double) * np * 4);
    int32_t *d_conn = (int32_t *)alloc(sizeof(int32_t) * ne * nv), *d_elem = (int32_t *)alloc(sizeof(int32_t) * np);
    unsigned long long *d_cnt = (unsigned long long *)alloc(8 * nb), *d_start = (unsigned long long *)alloc(8 * (nb + 1));
    unsigned long long *d_part = (unsigned long long *)alloc(8 * nparts), *d_fill = (unsigned long long *)alloc(8 * nb);
    if (!d_xyz || !d_f || !d_pts || !d_out || !d_lam || !d_conn || !d_elem || !d_cnt || !d_start || !d_part ||
        !d_fill) {
        release();
        return MLQ_ENOMEM;
    }
    bool ok = true;
    auto chk = [&](cudaError_t e) { ok = ok && e == cudaSuccess; };
    chk(cudaMemcpy(d_xyz, xyz, sizeof(double) * n * dim, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(d_f, f, sizeof(double) * n * K, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(d_pts, pts, sizeof(double) * np * dim, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(d_conn, conn, sizeof(int32_t) * ne * nv, cudaMemcpyHostToDevice));
    chk(cudaMemset(d_cnt, 0, 8 * nb));
    const LocMesh m{dim, n, ne, d_xyz, d_conn};
    const unsigned ge = (unsigned)((ne + kT - 1) / kT);
    if (ok) {
        box_count_kernel<<<ge, kT>>>(m, G, d_cnt);
        scan_local_kernel<<<(unsigned)nparts, kT>>>(nb, d_cnt, d_start, d_part);
        scan_parts_kernel<<<1, 32>>>(nparts, d_part, nb, d_start);
        scan_add_kernel<<<(unsigned)((nb + kT - 1) / kT), kT>>>(nb, d_part, d_start, d_fill);
        chk(cudaGetLastError());
    }
    unsigned long long total = 0;
    if (ok) chk(cudaMemcpy(&total, d_start + nb, 8, cudaMemcpyDeviceToHost));
    int32_t *d_list = ok ? (int32_t *)alloc(sizeof(int32_t) * std::max<unsigned long long>(total, 1)) : nullptr;
    if (ok && !d_list) {
        release();
        return MLQ_ENOMEM;
    }
    if (ok) {
        box_fill_kernel<<<ge, kT>>>(m, G, d_fill, d_list);
        locate_kernel<<<(unsigned)((np + kT - 1) / kT), kT>>>(m, G, d_start, d_list, np, d_pts, d_elem, d_lam);
        chk(cudaGetLastError());
    }
    // points in no simplex: the global scan, one CTA each
    std::vector<int32_t> elem(ok ? (size_t)np : 0);
    if (ok) chk(cudaMemcpy(elem.data(), d_elem, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    std::vector<int64_t> outside;
    for (int64_t p = 0; ok && p < np; ++p)
        if (elem[(size_t)p] < 0) outside.push_back(p);
    if (ok && !outside.empty()) {
        int64_t *d_which = (int64_t *)alloc(sizeof(int64_t) * outside.size());
        if (!d_which) {
            release();
            return MLQ_ENOMEM;
        }
        chk(cudaMemcpy(d_which, outside.data(), sizeof(int64_t) * outside.size(), cudaMemcpyHostToDevice));
        for (size_t c0 = 0; ok && c0 < outside.size(); c0 += 65535) {
            const unsigned nblk = (unsigned)std::min<size_t>(65535, outside.size() - c0);
            outside_kernel<<<nblk, kT>>>(m, d_pts, d_which + c0, d_elem, d_lam);
            chk(cudaGetLastError());
        }
    }
    if (ok) {
        interp_kernel<<<(unsigned)((np * K + kT - 1) / kT), kT>>>(m, K, d_f, np, d_elem, d_lam, d_out);
        chk(cudaGetLastError());
        chk(cudaMemcpy(out, d_out, sizeof(double) * np * K, cudaMemcpyDeviceToHost));
    }
    release();
    return ok ? MLQ_OK : MLQ_ECUDA;
}
