// mlq_mesh.cu -- levels on general tetrahedral meshes (non-nested
// hierarchies, Sec. 4 and Sec. 5.4): a first GPU member for meshes that are
// not structured boxes.
//
// Per sample s and time block, as for the structured levels (Sec. 3.1-3.3):
//   theta_e = theta_mean_e + sum_k Phi[e, k] xi_k                 (eq. KLlowrank)
//   f_e = cos(theta_e) e1_e + sin(theta_e) e2_e, D_e = s_t I + (s_l - s_t) f f^T
//                                                                 (eq. AdmV)
//   A = M + dt K(D) in CSR, b = M (v + dt R(v, w)), w += dt eps (v - gam w),
//   A v+ = b by Jacobi-preconditioned CG from v (FP64), Q = m^T v, m = M 1.
// The CSR values of A are gathered per nonzero over the element entries
// that add to it (a list fixed by the mesh), so every sum has a fixed order;
// dot products reduce per block in a fixed tree and then over blocks in
// order.  The CG iteration is driven from the host, one kernel per step
// with the samples batched; samples that have converged are frozen.
#include "mlq.h"

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

// y[s][i] = sum_t val[t (+ s nnz)] x[s][ci[t]]  (vs = 0: one matrix for all samples)
__global__ void spmv_kernel(int64_t n, int S, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ val, int64_t vs, const double *__restrict__ x,
                            double *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n || s >= S) return;
    const double *v = val + (int64_t)s * vs;
    const double *xs = x + (int64_t)s * n;
    double acc = 0.0;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) acc += v[t] * xs[ci[t]];
    y[(int64_t)s * n + i] = acc;
}

// per-block partial sums of u . v (fixed tree), part[s][blockIdx.x]
__global__ void dot_partial_kernel(int64_t n, int S, const double *__restrict__ u, const double *__restrict__ v,
                                   int64_t us, double *__restrict__ part)
{
    __shared__ double sh[kThreads];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    double x = 0.0;
    if (i < n && s < S) x = u[(int64_t)s * us + i] * v[(int64_t)s * n + i];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && s < S) part[(int64_t)s * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void dot_final_kernel(int S, int nb, const double *__restrict__ part, double *__restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[(int64_t)s * nb + b];
    out[s] = acc;
}

// y = v + dt R(v, w); w <- w + dt eps (v - gam w); x = v
__global__ void block_load_kernel(int64_t n, int S, double dt, double a, double eps, double gam,
                                  const double *__restrict__ v, double *__restrict__ w, double *__restrict__ y,
                                  double *__restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n || s >= S) return;
    const int64_t k = (int64_t)s * n + i;
    const double vv = v[k], ww = w[k];
    y[k] = vv + dt * (vv * (vv - a) * (1.0 - vv) - ww);
    w[k] = ww + dt * eps * (vv - gam * ww);
    x[k] = vv;
}

// r = b - q; z = dinv r; p = z
__global__ void cg_start_kernel(int64_t n, int S, const double *__restrict__ b, const double *__restrict__ q,
                                const double *__restrict__ dinv, double *__restrict__ r, double *__restrict__ z,
                                double *__restrict__ p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n || s >= S) return;
    const int64_t k = (int64_t)s * n + i;
    const double rr = b[k] - q[k];
    r[k] = rr;
    z[k] = dinv[k] * rr;
    p[k] = z[k];
}

// x += alpha p; r -= alpha q; z = dinv r
__global__ void cg_update_kernel(int64_t n, int S, const double *__restrict__ alpha, const double *__restrict__ p,
                                 const double *__restrict__ q, const double *__restrict__ dinv, double *__restrict__ x,
                                 double *__restrict__ r, double *__restrict__ z)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n || s >= S) return;
    const double al = alpha[s];
    if (al == 0.0) return;   // a sample that no longer iterates keeps x, r, z
    const int64_t k = (int64_t)s * n + i;
    x[k] += al * p[k];
    r[k] -= al * q[k];
    z[k] = dinv[k] * r[k];
}

__global__ void cg_direction_kernel(int64_t n, int S, const double *__restrict__ beta, const double *__restrict__ z,
                                    double *__restrict__ p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n || s >= S) return;
    const int64_t k = (int64_t)s * n + i;
    p[k] = z[k] + beta[s] * p[k];
}

__global__ void dinv_kernel(int64_t n, int S, int64_t nnz, const int64_t *__restrict__ diag,
                            const double *__restrict__ aval, double *__restrict__ dinv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n || s >= S) return;
    dinv[(int64_t)s * n + i] = 1.0 / aval[(int64_t)s * nnz + diag[i]];
}

// per-sample scalars of Jacobi-PCG.  st: 0 iterating, 1 converged, 2 iteration
// cap, 3 not finite.  Phase 0 (start): iterating iff ||r|| > tol ||b||.
// Phase 1 (after q = A p): alpha = rz / pq.  Phase 2 (after the update):
// convergence test and beta.  Phase 3: count the iterating samples only.
struct CgScalars {
    double *rz, *pq, *rr, *bb, *rzn, *alpha, *beta;
    int32_t *st, *it;
};

__global__ void cg_scalar_kernel(int S, int phase, double tol2, int64_t maxit, CgScalars c, int32_t *nactive)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    if (phase == 3) {
        if (nactive && c.st[s] == 0) atomicAdd(nactive, 1);
        return;
    }
    if (phase == 0) {
        c.st[s] = (c.rr[s] <= tol2 * c.bb[s]) ? 1 : 0;
        if (!isfinite(c.rr[s]) || !isfinite(c.bb[s])) c.st[s] = 3;
        c.alpha[s] = 0.0;
        c.beta[s] = 0.0;
    } else if (phase == 1) {
        const bool run = c.st[s] == 0 && c.pq[s] != 0.0 && isfinite(c.pq[s]);
        if (c.st[s] == 0 && !run) c.st[s] = isfinite(c.pq[s]) ? 1 : 3;
        c.alpha[s] = run ? c.rz[s] / c.pq[s] : 0.0;
    } else {
        c.beta[s] = 0.0;
        if (c.st[s] == 0) {
            c.it[s] += 1;
            if (!isfinite(c.rr[s])) c.st[s] = 3;
            else if (c.rr[s] <= tol2 * c.bb[s]) c.st[s] = 1;
            else if (c.it[s] >= maxit) c.st[s] = 2;
            if (c.st[s] == 0) c.beta[s] = c.rzn[s] / c.rz[s];
            c.rz[s] = c.rzn[s];
        }
    }
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

int mlq_mesh_solve(mlq_mesh *m, const mlq_model *model, double dt, int32_t nsteps, double rtol, const double *v0,
                   const double *w0, int64_t S, const double *xi, double *q_out, int32_t *status, int32_t *iters)
{
    if (!m || !model || !(dt > 0.0) || nsteps < 0 || !(rtol > 0.0) || !v0 || S < 0 || S > 65535 || !q_out)
        return MLQ_EINVAL;
    if (S == 0) return MLQ_OK;
    if (m->K > 0 && !xi) return MLQ_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return MLQ_ECUDA;
    const int64_t n = m->n, ne = m->ne, nnz = m->nnz, sn = S * n;
    const int nbn = (int)((n + kThreads - 1) / kThreads);
    std::vector<void *> allocs;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 8)) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return p;
    };
    auto release = [&]() {
        for (void *p : allocs) cudaFree(p);
    };
    double *cs2 = (double *)alloc((size_t)S * ne * 2 * 8), *aval = (double *)alloc((size_t)S * nnz * 8);
    double *dinv = (double *)alloc(sn * 8), *v = (double *)alloc(sn * 8), *w = (double *)alloc(sn * 8);
    double *y = (double *)alloc(sn * 8), *b = (double *)alloc(sn * 8), *x = (double *)alloc(sn * 8);
    double *r = (double *)alloc(sn * 8), *z = (double *)alloc(sn * 8), *p = (double *)alloc(sn * 8);
    double *q = (double *)alloc(sn * 8), *part = (double *)alloc((size_t)S * nbn * 8);
    double *xi_d = (double *)alloc((size_t)S * std::max(m->K, 1) * 8);
    double *sc = (double *)alloc((size_t)S * 7 * 8);
    int32_t *si = (int32_t *)alloc((size_t)S * 2 * 4), *nact = (int32_t *)alloc(4);
    if (!cs2 || !aval || !dinv || !v || !w || !y || !b || !x || !r || !z || !p || !q || !part || !xi_d || !sc || !si ||
        !nact) {
        release();
        return MLQ_ENOMEM;
    }
    CgScalars c{sc, sc + S, sc + 2 * S, sc + 3 * S, sc + 4 * S, sc + 5 * S, sc + 6 * S, si, si + S};
    bool ok = true;
    auto chk = [&](cudaError_t e) { ok = ok && e == cudaSuccess; };
    if (m->K > 0) chk(cudaMemcpy(xi_d, xi, (size_t)S * m->K * 8, cudaMemcpyHostToDevice));
    // initial state for every sample
    for (int64_t s = 0; s < S && ok; ++s) {
        chk(cudaMemcpy(v + s * n, v0, (size_t)n * 8, cudaMemcpyHostToDevice));
        if (w0) chk(cudaMemcpy(w + s * n, w0, (size_t)n * 8, cudaMemcpyHostToDevice));
        else chk(cudaMemset(w + s * n, 0, (size_t)n * 8));
    }
    chk(cudaMemset(si, 0, (size_t)S * 2 * 4));
    const dim3 ge((unsigned)((ne + kThreads - 1) / kThreads), (unsigned)S), gz((unsigned)((nnz + kThreads - 1) / kThreads), (unsigned)S);
    const dim3 gn((unsigned)nbn, (unsigned)S);
    const unsigned gs = (unsigned)((S + 127) / 128);
    synth_kernel<<<ge, kThreads>>>(m->phi, m->theta_mean, xi_d, m->K, ne, (int)S, cs2);
    assemble_kernel<<<gz, kThreads>>>(nnz, (int)S, m->cstart, m->centry, m->geo, m->frames, cs2, ne, model->s_l,
                                      model->s_t, dt, m->mval, aval);
    dinv_kernel<<<gn, kThreads>>>(n, (int)S, nnz, m->diag, aval, dinv);
    chk(cudaGetLastError());
    auto dot = [&](const double *u, int64_t us, const double *vv, double *outp) {
        dot_partial_kernel<<<gn, kThreads>>>(n, (int)S, u, vv, us, part);
        dot_final_kernel<<<gs, 128>>>((int)S, nbn, part, outp);
    };
    const int64_t maxit = 10 * n;
    const double tol2 = rtol * rtol;
    std::vector<int32_t> it_total((size_t)S, 0), st_worst((size_t)S, 0), it_h((size_t)S), st_h((size_t)S);
    for (int32_t step = 0; step < nsteps && ok; ++step) {
        block_load_kernel<<<gn, kThreads>>>(n, (int)S, dt, model->a, model->eps, model->gamma, v, w, y, x);
        spmv_kernel<<<gn, kThreads>>>(n, (int)S, m->rp, m->ci, m->mval, 0, y, b);      // b = M y
        spmv_kernel<<<gn, kThreads>>>(n, (int)S, m->rp, m->ci, aval, nnz, x, q);       // q = A x
        cg_start_kernel<<<gn, kThreads>>>(n, (int)S, b, q, dinv, r, z, p);
        dot(r, n, z, c.rz);
        dot(r, n, r, c.rr);
        dot(b, n, b, c.bb);
        chk(cudaMemset(c.it, 0, (size_t)S * 4));
        cg_scalar_kernel<<<gs, 128>>>((int)S, 0, tol2, maxit, c, nullptr);
        for (int64_t k = 0; ok; ++k) {
            if (k % 4 == 0) {
                chk(cudaMemset(nact, 0, 4));
                cg_scalar_kernel<<<gs, 128>>>((int)S, 3, tol2, maxit, c, nact);
                int32_t na = 0;
                chk(cudaMemcpy(&na, nact, 4, cudaMemcpyDeviceToHost));
                if (na == 0) break;
            }
            spmv_kernel<<<gn, kThreads>>>(n, (int)S, m->rp, m->ci, aval, nnz, p, q);   // q = A p
            dot(p, n, q, c.pq);
            cg_scalar_kernel<<<gs, 128>>>((int)S, 1, tol2, maxit, c, nullptr);
            cg_update_kernel<<<gn, kThreads>>>(n, (int)S, c.alpha, p, q, dinv, x, r, z);
            dot(r, n, z, c.rzn);
            dot(r, n, r, c.rr);
            cg_scalar_kernel<<<gs, 128>>>((int)S, 2, tol2, maxit, c, nullptr);
            cg_direction_kernel<<<gn, kThreads>>>(n, (int)S, c.beta, z, p);
            chk(cudaGetLastError());
        }
        chk(cudaMemcpy(v, x, (size_t)sn * 8, cudaMemcpyDeviceToDevice));
        chk(cudaMemcpy(it_h.data(), c.it, (size_t)S * 4, cudaMemcpyDeviceToHost));
        chk(cudaMemcpy(st_h.data(), c.st, (size_t)S * 4, cudaMemcpyDeviceToHost));
        for (int64_t s = 0; s < S; ++s) {
            it_total[(size_t)s] += it_h[(size_t)s];
            const int32_t code = st_h[(size_t)s] == 1 ? MLQ_S_CONVERGED
                                 : (st_h[(size_t)s] == 2 ? MLQ_S_MAXITER : (st_h[(size_t)s] == 3 ? MLQ_S_NONFINITE : MLQ_S_MAXITER));
            st_worst[(size_t)s] = std::max(st_worst[(size_t)s], code);
        }
    }
    // Q = m^T v
    if (ok) {
        dot(m->lump, 0, v, c.rz);
        chk(cudaMemcpy(q_out, c.rz, (size_t)S * 8, cudaMemcpyDeviceToHost));
        chk(cudaDeviceSynchronize());
    }
    release();
    if (!ok) return MLQ_ECUDA;
    for (int64_t s = 0; s < S; ++s) {
        if (status) status[s] = st_worst[(size_t)s];
        if (iters) iters[s] = it_total[(size_t)s];
    }
    return MLQ_OK;
}

}  // extern "C"
