// mlq_mesh.cu -- levels on general tetrahedral meshes (non-nested
// hierarchies, Sec. 4 and Sec. 5.4): the GPU member for meshes that are not
// structured boxes, standalone (mlq_mesh_*) or as a level of a context
// (mlq_add_level_mesh, through mlq_mesh_member.h).
//
// Per sample s and time block, as for the structured levels (Sec. 3.1-3.3):
//   theta_e = theta_mean_e + sum_k Phi[e, k] xi_k                 (eq. KLlowrank)
//   f_e = cos(theta_e) e1_e + sin(theta_e) e2_e, D_e = s_t I + (s_l - s_t) f f^T
//                                                                 (eq. AdmV)
//   A = M + dt K(D) in CSR, b = M (v + dt R(v, w)), w += dt eps (v - gam w),
//   A v+ = b by Jacobi-preconditioned CG from v (FP64), Q = m^T v, m = M 1.
// The CSR values of A are gathered per nonzero over the element entries
// that add to it (a list fixed by the mesh), so every sum has a fixed order.
// The time blocks run in one launch of mesh_slab_kernel (mlq_mesh_solver.cuh):
// one sample per cluster of CTAs, or per group of many CTAs in one
// cooperative launch (mlq_groups.cuh), FP64 Jacobi-PCG or FP32 inner PCG
// inside FP64 refinement, with no host synchronisation inside the solve.
#include "mlq.h"
#include "mlq_launch.cuh"
#include "mlq_mesh_member.h"
#include "mlq_mesh_solver.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

namespace {

constexpr int kThreads = 256;

__global__ void synth_kernel(const double *__restrict__ phi, const double *__restrict__ theta_mean,
                             const double *__restrict__ xi, int K, int64_t ne, int S, double *__restrict__ cs2)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (e >= ne || s >= S) return;
    double t = theta_mean ? theta_mean[e] : 0.0;
    for (int k = 0; k < K; ++k) t += phi[e * K + k] * xi[(int64_t)s * K + k];
    cs2[((int64_t)s * ne + e) * 2] = cos(2.0 * t);
    cs2[((int64_t)s * ne + e) * 2 + 1] = sin(2.0 * t);
}

// a[s][t] = mval[t] + dt sum over the entries (e, a, b) of nonzero t of
// |e| grad_a^T D_e grad_b; D_e from (cos 2 theta, sin 2 theta) and the frame:
// f f^T = ((1 + c) e1 e1^T + (1 - c) e2 e2^T + sn (e1 e2^T + e2 e1^T)) / 2
__global__ void assemble_kernel(int64_t nnz, int S, const int64_t *__restrict__ cstart,
                                const int32_t *__restrict__ centry, const double *__restrict__ geo,
                                const double *__restrict__ frames, const double *__restrict__ cs2, int64_t ne,
                                double s_l, double s_t, double dt, const double *__restrict__ mval,
                                double *__restrict__ aval)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (t >= nnz || s >= S) return;
    double acc = 0.0;
    for (int64_t c = cstart[t]; c < cstart[t + 1]; ++c) {
        const int32_t ent = centry[c];
        const int64_t e = ent >> 4;
        const int a = (ent >> 2) & 3, b = ent & 3;
        const double cc = cs2[((int64_t)s * ne + e) * 2], sn = cs2[((int64_t)s * ne + e) * 2 + 1];
        const double *f = frames + e * 6;
        double D[3][3];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q)
                D[r][q] = (r == q ? s_t : 0.0) +
                          0.5 * (s_l - s_t) *
                              ((1.0 + cc) * f[r] * f[q] + (1.0 - cc) * f[3 + r] * f[3 + q] +
                               sn * (f[r] * f[3 + q] + f[3 + r] * f[q]));
        const double *ga = geo + e * 13 + a * 3, *gb = geo + e * 13 + b * 3;
        double k = 0.0;
        for (int r = 0; r < 3; ++r) k += ga[r] * (D[r][0] * gb[0] + D[r][1] * gb[1] + D[r][2] * gb[2]);
        acc += geo[e * 13 + 12] * k;
    }
    aval[(int64_t)s * nnz + t] = mval[t] + dt * acc;
}

// FP32 copy of the CSR values (the mixed path's inner matrix)
__global__ void to_f32_kernel(int64_t count, const double *__restrict__ a, float *__restrict__ f)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) f[t] = (float)a[t];
}

struct Csr {
    std::vector<int64_t> rp, cstart, diag;
    std::vector<int32_t> ci, centry;
};

// pattern of the P1 matrices (i, j share a tetrahedron), and per nonzero the
// element entries (e, a, b) that add to it, in element order
void build_csr(int64_t n, int64_t ne, const int32_t *conn, Csr &C)
{
    std::vector<std::vector<int32_t>> rows((size_t)n);
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) rows[(size_t)conn[e * 4 + a]].push_back(conn[e * 4 + b]);
    C.rp.assign((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        std::vector<int32_t> &r = rows[(size_t)i];
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        C.rp[(size_t)i + 1] = C.rp[(size_t)i] + (int64_t)r.size();
    }
    C.ci.resize((size_t)C.rp[(size_t)n]);
    C.diag.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        std::copy(rows[(size_t)i].begin(), rows[(size_t)i].end(), C.ci.begin() + C.rp[(size_t)i]);
        const auto it = std::lower_bound(rows[(size_t)i].begin(), rows[(size_t)i].end(), (int32_t)i);
        C.diag[(size_t)i] = C.rp[(size_t)i] + (it - rows[(size_t)i].begin());
        std::vector<int32_t>().swap(rows[(size_t)i]);
    }
    const int64_t nnz = C.rp[(size_t)n];
    auto pos = [&](int32_t i, int32_t j) {
        const auto b = C.ci.begin() + C.rp[(size_t)i], e = C.ci.begin() + C.rp[(size_t)i + 1];
        return (int64_t)(std::lower_bound(b, e, j) - C.ci.begin());
    };
    C.cstart.assign((size_t)nnz + 1, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) ++C.cstart[(size_t)pos(conn[e * 4 + a], conn[e * 4 + b]) + 1];
    for (int64_t t = 0; t < nnz; ++t) C.cstart[(size_t)t + 1] += C.cstart[(size_t)t];
    C.centry.resize((size_t)C.cstart[(size_t)nnz]);
    std::vector<int64_t> fill(C.cstart.begin(), C.cstart.end() - 1);
    for (int64_t e = 0; e < ne; ++e)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                C.centry[(size_t)fill[(size_t)pos(conn[e * 4 + a], conn[e * 4 + b])]++] = (int32_t)(e * 16 + a * 4 + b);
}

template <typename T>
T *dev_copy(const T *h, size_t count)
{
    T *d = nullptr;
    if (cudaMalloc(&d, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    if (count && cudaMemcpy(d, h, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    return d;
}

}  // namespace

struct mlq_mesh {
    int device = 0;
    int64_t n = 0, ne = 0, nnz = 0;
    int K = 0;
    int64_t *rp = nullptr, *cstart = nullptr, *diag = nullptr;
    int32_t *ci = nullptr, *centry = nullptr;
    double *geo = nullptr, *frames = nullptr, *mval = nullptr, *lump = nullptr;
    double *phi = nullptr, *theta_mean = nullptr;
    std::vector<double> lump_h;
};

namespace {

template <typename TI>
mlq::MeshArgs<TI> mesh_args(const mlq_mesh *m, const mlq_model *model, const mlq_options &o, double dt, int nsteps,
                            int64_t S, const double *aval, const TI *ai, const double *v0, const double *w0,
                            double *v, double *w, double *b, double *y, void *const *vec, double *q, int32_t *it,
                            int32_t *st)
{
    mlq::MeshArgs<TI> a{};
    a.n = (int)m->n;
    a.S = (int)S;
    a.nnz = m->nnz;
    a.rp = m->rp;
    a.ci = m->ci;
    a.diag = m->diag;
    a.mval = m->mval;
    a.lump = m->lump;
    a.A64 = aval;
    a.Ai = ai;
    a.dt = dt;
    a.nsteps = nsteps;
    a.a = model->a;
    a.eps = model->eps;
    a.gam = model->gamma;
    a.rtol_out = o.rtol;
    a.rtol_in = o.rtol_inner;
    a.max_iter = o.max_iter;
    a.max_sweeps = o.max_sweeps;
    a.v0 = v0;
    a.w0 = w0;
    a.v = v;
    a.w = w;
    a.b = b;
    a.y = y;
    a.r = (TI *)vec[0];
    a.u = (TI *)vec[1];
    a.wv = (TI *)vec[2];
    a.s = (TI *)vec[3];
    a.p = (TI *)vec[4];
    a.x = (TI *)vec[5];
    a.dinv = (TI *)vec[6];
    a.q = q;
    a.iters = it;
    a.status = st;
    return a;
}

constexpr int kMeshThreads = 512;

template <typename TI, bool PTS>
cudaError_t launch_mesh_t(int cs, const mlq::MeshArgs<TI> &a, cudaStream_t st)
{
    switch (cs) {
    case 1: return mlq::cluster_launch<1>(mlq::mesh_slab_kernel<TI, mlq::ClusterGroup<1>, PTS>, a.S, kMeshThreads, 0, st, a, mlq::ClusterGroup<1>{});
    case 2: return mlq::cluster_launch<2>(mlq::mesh_slab_kernel<TI, mlq::ClusterGroup<2>, PTS>, a.S, kMeshThreads, 0, st, a, mlq::ClusterGroup<2>{});
    case 4: return mlq::cluster_launch<4>(mlq::mesh_slab_kernel<TI, mlq::ClusterGroup<4>, PTS>, a.S, kMeshThreads, 0, st, a, mlq::ClusterGroup<4>{});
    case 8: return mlq::cluster_launch<8>(mlq::mesh_slab_kernel<TI, mlq::ClusterGroup<8>, PTS>, a.S, kMeshThreads, 0, st, a, mlq::ClusterGroup<8>{});
    case 16: return mlq::cluster_launch<16>(mlq::mesh_slab_kernel<TI, mlq::ClusterGroup<16>, PTS>, a.S, kMeshThreads, 0, st, a, mlq::ClusterGroup<16>{});
    default: return cudaErrorInvalidValue;
    }
}

// the instantiation with point QoIs only when the launch records points
template <typename TI>
cudaError_t launch_mesh(int cs, const mlq::MeshArgs<TI> &a, cudaStream_t st)
{
    return a.pq.npts > 0 ? launch_mesh_t<TI, true>(cs, a, st) : launch_mesh_t<TI, false>(cs, a, st);
}

// G CTAs per sample in one cooperative launch (every CTA resident at once:
// the launch fails otherwise)
template <typename TI>
cudaError_t launch_mesh_grid(const mlq::MeshArgs<TI> &a, const mlq::GridGroup &grp, cudaStream_t st)
{
    auto kern = a.pq.npts > 0 ? mlq::mesh_slab_kernel<TI, mlq::GridGroup, true>
                              : mlq::mesh_slab_kernel<TI, mlq::GridGroup, false>;
    int prio = 0;
    cudaError_t e = cudaStreamGetPriority(st, &prio);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(a.S * grp.G));
    cfg.blockDim = dim3((unsigned)kMeshThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributePriority;
    attr[1].val.priority = prio;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, a, grp);
}

// CTAs of the mesh kernel resident at once on the device (every variant
// has the same bounds; the smallest count decides)
int64_t mesh_resident_ctas(int device)
{
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    void (*const kerns[2])(mlq::MeshArgs<float>, mlq::GridGroup) = {
        mlq::mesh_slab_kernel<float, mlq::GridGroup, false>, mlq::mesh_slab_kernel<float, mlq::GridGroup, true>};
    void (*const kerns64[2])(mlq::MeshArgs<double>, mlq::GridGroup) = {
        mlq::mesh_slab_kernel<double, mlq::GridGroup, false>, mlq::mesh_slab_kernel<double, mlq::GridGroup, true>};
    int best = 1 << 30;
    for (int k = 0; k < 2; ++k) {
        int b32 = 0, b64 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, kerns[k], kMeshThreads, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, kerns64[k], kMeshThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        best = std::min(best, std::min(b32, b64));
    }
    return (int64_t)best * nsm;
}

size_t align256(size_t b) { return (std::max<size_t>(b, 8) + 255) / 256 * 256; }

}  // namespace

namespace mlq {

int64_t mesh_nodes(const mlq_mesh *m) { return m->n; }
int64_t mesh_elems(const mlq_mesh *m) { return m->ne; }
int mesh_modes(const mlq_mesh *m) { return m->K; }

MeshShape mesh_member_shape(const mlq_mesh *m, int64_t S, int request)
{
    MeshShape sh;
    S = std::max<int64_t>(S, 1);
    if (request > 16) {
        sh.G = request;
        sh.cs = (int64_t)request * S <= mesh_resident_ctas(m->device) ? 1 : 0;
        return sh;
    }
    if (request > 0) {
        while (sh.cs * 2 <= request) sh.cs *= 2;
        while (sh.cs > 1 && m->n / sh.cs < 64) sh.cs /= 2;
        return sh;
    }
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    // one cluster of 16 per sample leaves SMs idle: spread each sample over
    // up to min(resident CTAs / S, n / 2048) CTAs; when that many CTAs
    // outnumber the SMs, take k SMs' worth (k = 2, else 1) so that every SM
    // holds the same number of CTAs and no barrier waits for a CTA that
    // shares its SM
    const int64_t res = mesh_resident_ctas(m->device);
    if (16 * S < 2LL * nsm) {
        const int64_t cap = std::min<int64_t>(res / S, m->n / 2048);
        int64_t G = cap;
        if (cap * S > nsm) G = 2LL * nsm / S <= cap ? 2LL * nsm / S : nsm / S;
        if (G > 16) {
            sh.G = (int)G;
            return sh;
        }
    }
    while (sh.cs < 16 && (int64_t)(2 * sh.cs) * S <= 2LL * nsm && m->n / (2 * sh.cs) >= 4096) sh.cs *= 2;
    while (sh.cs > 1 && m->n / sh.cs < 64) sh.cs /= 2;
    return sh;
}

size_t mesh_member_bytes(const mlq_mesh *m, bool mixed, int64_t S, const MeshShape &sh)
{
    const size_t sn = (size_t)S * m->n, ti = mixed ? 4 : 8;
    size_t t = align256((size_t)S * m->ne * 16) + align256((size_t)S * m->nnz * 8);
    if (mixed) t += align256((size_t)S * m->nnz * 4);
    t += 4 * align256(sn * 8) + 7 * align256(sn * ti);
    t += align256((size_t)S * 8) + 2 * align256((size_t)S * 4);
    if (sh.G > 0) t += align256((size_t)S * 2 * sizeof(unsigned)) + align256((size_t)S * 2 * sh.G * 4 * 8);
    return t;
}

MeshWs mesh_member_carve(const mlq_mesh *m, bool mixed, int64_t S, const MeshShape &sh, char *&base)
{
    const size_t sn = (size_t)S * m->n, ti = mixed ? 4 : 8;
    auto take = [&](size_t bytes) {
        char *p = base;
        base += align256(bytes);
        return (void *)p;
    };
    MeshWs w;
    w.cs2 = (double *)take((size_t)S * m->ne * 16);
    w.aval = (double *)take((size_t)S * m->nnz * 8);
    w.a32 = mixed ? (float *)take((size_t)S * m->nnz * 4) : nullptr;
    w.v = (double *)take(sn * 8);
    w.w = (double *)take(sn * 8);
    w.b = (double *)take(sn * 8);
    w.y = (double *)take(sn * 8);
    for (void *&p : w.vec) p = take(sn * ti);
    w.q = (double *)take((size_t)S * 8);
    w.iters = (int32_t *)take((size_t)S * 4);
    w.status = (int32_t *)take((size_t)S * 4);
    if (sh.G > 0) {
        w.bar = (unsigned *)take((size_t)S * 2 * sizeof(unsigned));
        w.part = (double *)take((size_t)S * 2 * sh.G * 4 * 8);
    }
    return w;
}

cudaError_t mesh_member_launch(const mlq_mesh *m, const mlq_model &model, const mlq_options &opt, double dt,
                               int nsteps, const double *d_v0, const double *d_w0, int64_t S, const double *d_xi,
                               const MeshWs &ws, const MeshShape &sh, int *err, cudaStream_t st, bool setup,
                               bool solve, const PointArgs *points)
{
    if (sh.cs < 1 || (sh.G > 0 && (!ws.bar || !ws.part || !err))) return cudaErrorInvalidValue;
    if (S <= 0) return cudaSuccess;
    const bool mixed = opt.precision == MLQ_MIXED;
    const int64_t ne = m->ne, nnz = m->nnz;
    if (setup) {
        const dim3 ge((unsigned)((ne + kThreads - 1) / kThreads), (unsigned)S);
        const dim3 gz((unsigned)((nnz + kThreads - 1) / kThreads), (unsigned)S);
        synth_kernel<<<ge, kThreads, 0, st>>>(m->phi, m->theta_mean, d_xi, m->K, ne, (int)S, ws.cs2);
        assemble_kernel<<<gz, kThreads, 0, st>>>(nnz, (int)S, m->cstart, m->centry, m->geo, m->frames, ws.cs2, ne,
                                                 model.s_l, model.s_t, dt, m->mval, ws.aval);
        if (mixed)
            to_f32_kernel<<<(unsigned)((S * nnz + kThreads - 1) / kThreads), kThreads, 0, st>>>(S * nnz, ws.aval,
                                                                                               ws.a32);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!solve) return cudaSuccess;
    mlq::GridGroup grp{sh.G, ws.bar, ws.part, err};
    if (sh.G > 0) {
        const cudaError_t e = cudaMemsetAsync(ws.bar, 0, (size_t)S * 2 * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
    }
    const PointArgs pq = points ? *points : PointArgs{0, nullptr, nullptr, 0.0, nullptr, nullptr};
    if (mixed) {
        mlq::MeshArgs<float> a = mesh_args<float>(m, &model, opt, dt, nsteps, S, ws.aval, ws.a32, d_v0, d_w0, ws.v, ws.w,
                                                  ws.b, ws.y, ws.vec, ws.q, ws.iters, ws.status);
        a.pq = pq;
        return sh.G > 0 ? launch_mesh_grid<float>(a, grp, st) : launch_mesh<float>(sh.cs, a, st);
    }
    mlq::MeshArgs<double> a = mesh_args<double>(m, &model, opt, dt, nsteps, S, ws.aval, ws.aval, d_v0, d_w0, ws.v, ws.w,
                                                ws.b, ws.y, ws.vec, ws.q, ws.iters, ws.status);
    a.pq = pq;
    return sh.G > 0 ? launch_mesh_grid<double>(a, grp, st) : launch_mesh<double>(sh.cs, a, st);
}

}  // namespace mlq

extern "C" {

int mlq_mesh_create(mlq_mesh **out, int device, int64_t n, const double *xyz, int64_t ne, const int32_t *conn,
                    const double *frames)
{
    if (!out || n < 4 || ne < 1 || !xyz || !conn || ne > ((int64_t)1 << 27)) return MLQ_EINVAL;
    for (int64_t t = 0; t < ne * 4; ++t)
        if (conn[t] < 0 || conn[t] >= n) return MLQ_EINVAL;
    *out = nullptr;
    try {
        if (cudaSetDevice(device) != cudaSuccess) return MLQ_ECUDA;
        mlq_mesh *m = new mlq_mesh();
        m->device = device;
        m->n = n;
        m->ne = ne;
        // geometry per tetrahedron: gradients of the barycentric functions
        // (4 x 3) and the volume
        std::vector<double> geo((size_t)ne * 13);
        for (int64_t e = 0; e < ne; ++e) {
            const double *P[4];
            for (int a = 0; a < 4; ++a) P[a] = xyz + (int64_t)conn[e * 4 + a] * 3;
            double J[3][3];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) J[r][c] = P[c + 1][r] - P[0][r];   // columns: edges from vertex 0
            const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            if (!(std::fabs(det) > 0.0)) {
                delete m;
                return MLQ_EINVAL;
            }
            // rows of J^{-1} are the gradients of lambda_1..lambda_3
            double Ji[3][3];
            Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
            Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
            Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
            Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
            Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
            Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
            Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
            Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
            Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
            double *g = geo.data() + e * 13;
            for (int c = 0; c < 3; ++c) {
                g[3 + c] = Ji[0][c];
                g[6 + c] = Ji[1][c];
                g[9 + c] = Ji[2][c];
                g[c] = -(Ji[0][c] + Ji[1][c] + Ji[2][c]);
            }
            g[12] = std::fabs(det) / 6.0;
        }
        Csr C;
        build_csr(n, ne, conn, C);
        m->nnz = C.rp[(size_t)n];
        // consistent mass (|e| (1 + delta_ab) / 20) and its row sums
        std::vector<double> mval((size_t)m->nnz, 0.0);
        for (int64_t t = 0; t < m->nnz; ++t)
            for (int64_t c = C.cstart[(size_t)t]; c < C.cstart[(size_t)t + 1]; ++c) {
                const int32_t ent = C.centry[(size_t)c];
                const int64_t e = ent >> 4;
                const int a = (ent >> 2) & 3, b = ent & 3;
                mval[(size_t)t] += geo[(size_t)e * 13 + 12] / 20.0 * (a == b ? 2.0 : 1.0);
            }
        m->lump_h.assign((size_t)n, 0.0);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t t = C.rp[(size_t)i]; t < C.rp[(size_t)i + 1]; ++t) m->lump_h[(size_t)i] += mval[(size_t)t];
        std::vector<double> fr((size_t)ne * 6);
        for (int64_t e = 0; e < ne; ++e)
            for (int c = 0; c < 6; ++c) fr[(size_t)e * 6 + c] = frames ? frames[e * 6 + c] : (c == 0 || c == 4 ? 1.0 : 0.0);
        m->rp = dev_copy(C.rp.data(), C.rp.size());
        m->ci = dev_copy(C.ci.data(), C.ci.size());
        m->diag = dev_copy(C.diag.data(), C.diag.size());
        m->cstart = dev_copy(C.cstart.data(), C.cstart.size());
        m->centry = dev_copy(C.centry.data(), C.centry.size());
        m->geo = dev_copy(geo.data(), geo.size());
        m->frames = dev_copy(fr.data(), fr.size());
        m->mval = dev_copy(mval.data(), mval.size());
        m->lump = dev_copy(m->lump_h.data(), m->lump_h.size());
        if (!m->rp || !m->ci || !m->diag || !m->cstart || !m->centry || !m->geo || !m->frames || !m->mval || !m->lump) {
            mlq_mesh_destroy(m);
            return MLQ_ENOMEM;
        }
        *out = m;
        return MLQ_OK;
    } catch (...) {
        return MLQ_ENOMEM;
    }
}

int mlq_mesh_destroy(mlq_mesh *m)
{
    if (!m) return MLQ_OK;
    cudaSetDevice(m->device);
    for (void *p : {(void *)m->rp, (void *)m->ci, (void *)m->diag, (void *)m->cstart, (void *)m->centry,
                    (void *)m->geo, (void *)m->frames, (void *)m->mval, (void *)m->lump, (void *)m->phi,
                    (void *)m->theta_mean})
        if (p) cudaFree(p);
    delete m;
    return MLQ_OK;
}

int mlq_mesh_set_kl(mlq_mesh *m, int K, const double *phi, const double *theta_mean)
{
    if (!m || K < 0 || K > 4096 || (K > 0 && !phi)) return MLQ_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return MLQ_ECUDA;
    if (m->phi) cudaFree(m->phi);
    if (m->theta_mean) cudaFree(m->theta_mean);
    m->phi = m->theta_mean = nullptr;
    m->K = K;
    if (K > 0 && !(m->phi = dev_copy(phi, (size_t)m->ne * K))) return MLQ_ENOMEM;
    if (theta_mean && !(m->theta_mean = dev_copy(theta_mean, (size_t)m->ne))) return MLQ_ENOMEM;
    return MLQ_OK;
}

int mlq_mesh_solve_opts(mlq_mesh *m, const mlq_model *model, const mlq_options *opt, double dt, int32_t nsteps,
                        const double *v0, const double *w0, int64_t S, const double *xi, double *q_out,
                        int32_t *status, int32_t *iters)
{
    if (!m || !model || !opt || !(dt > 0.0) || nsteps < 0 || !v0 || S < 0 || S > 65535 || !q_out) return MLQ_EINVAL;
    if (opt->precision != MLQ_FP64 && opt->precision != MLQ_MIXED) return MLQ_EINVAL;
    if (!(opt->rtol > 0.0) || opt->max_iter < 1 || (opt->precision == MLQ_MIXED && opt->max_sweeps < 1))
        return MLQ_EINVAL;
    if (!(opt->cluster == 0 || opt->cluster == 1 || opt->cluster == 2 || opt->cluster == 4 || opt->cluster == 8 ||
          (opt->cluster >= 16 && opt->cluster <= 4096)))
        return MLQ_EINVAL;
    if (S == 0) return MLQ_OK;
    if (m->K > 0 && !xi) return MLQ_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return MLQ_ECUDA;
    const bool mixed = opt->precision == MLQ_MIXED;
    const int64_t n = m->n;
    const mlq::MeshShape sh = mlq::mesh_member_shape(m, S, opt->cluster);
    if (sh.cs < 1) return MLQ_EUNSUPPORTED;   // the requested CTAs cannot all be resident
    const size_t ws_b = mlq::mesh_member_bytes(m, mixed, S, sh) + align256(sizeof(int));
    const size_t in_b = align256((size_t)S * std::max(m->K, 1) * 8) + 2 * align256((size_t)n * 8);
    char *blk = nullptr;
    if (cudaMalloc(&blk, ws_b + in_b) != cudaSuccess) {
        cudaGetLastError();
        return MLQ_ENOMEM;
    }
    char *cur = blk;
    const mlq::MeshWs ws = mlq::mesh_member_carve(m, mixed, S, sh, cur);
    int *err_d = (int *)cur;
    cur += align256(sizeof(int));
    double *xi_d = (double *)cur;
    cur += align256((size_t)S * std::max(m->K, 1) * 8);
    double *v0_d = (double *)cur;
    cur += align256((size_t)n * 8);
    double *w0_d = w0 ? (double *)cur : nullptr;
    bool ok = true;
    auto chk = [&](cudaError_t e) { ok = ok && e == cudaSuccess; };
    if (m->K > 0) chk(cudaMemcpy(xi_d, xi, (size_t)S * m->K * 8, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(v0_d, v0, (size_t)n * 8, cudaMemcpyHostToDevice));
    if (w0) chk(cudaMemcpy(w0_d, w0, (size_t)n * 8, cudaMemcpyHostToDevice));
    int herr = 0;
    if (ok) {
        chk(cudaMemset(err_d, 0, sizeof(int)));
        chk(mlq::mesh_member_launch(m, *model, *opt, dt, nsteps, v0_d, w0_d, S, xi_d, ws, sh, err_d, nullptr));
        chk(cudaMemcpy(q_out, ws.q, (size_t)S * 8, cudaMemcpyDeviceToHost));
        if (status) chk(cudaMemcpy(status, ws.status, (size_t)S * 4, cudaMemcpyDeviceToHost));
        if (iters) chk(cudaMemcpy(iters, ws.iters, (size_t)S * 4, cudaMemcpyDeviceToHost));
        chk(cudaMemcpy(&herr, err_d, sizeof(int), cudaMemcpyDeviceToHost));
        chk(cudaDeviceSynchronize());
    }
    cudaFree(blk);
    if (!ok) return MLQ_ECUDA;
    return herr ? MLQ_ETIMEOUT : MLQ_OK;
}

int mlq_mesh_solve(mlq_mesh *m, const mlq_model *model, double dt, int32_t nsteps, double rtol, const double *v0,
                   const double *w0, int64_t S, const double *xi, double *q_out, int32_t *status, int32_t *iters)
{
    if (!m) return MLQ_EINVAL;
    mlq_options o;
    mlq_default_options(&o, MLQ_FP64);
    o.rtol = rtol;
    o.max_iter = (int)std::min<int64_t>(10 * m->n, 0x7fffffff);
    return mlq_mesh_solve_opts(m, model, &o, dt, nsteps, v0, w0, S, xi, q_out, status, iters);
}

}  // extern "C"
