// mlq_api.cu -- host runtime and C ABI of libmlq (see include/mlq.h).
//
// A context owns: the model and solver options, the level table (structured
// meshes of the nested hierarchy, KL mode tables in device memory, launch
// shapes), a device workspace that grows on demand, and a small pool of
// CUDA streams on which the members of a multilevel estimate run
// concurrently.  All compute happens in the kernels of mlq_kernels.cuh.
#include "mlq.h"
#include "mlq_aux.cuh"
#include "mlq_kl_tc.cuh"
#include "mlq_launch.cuh"
#include "mlq_host.h"
#include "mlq_mesh_member.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <mutex>
#include <thread>
#include <vector>

namespace {

constexpr int kMaxLevels = 16;
constexpr int kMaxK = 256;
constexpr int kStreams = 12;
// concurrent member streams of an estimate: the device's default number of
// hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS); more streams share one
constexpr int kLanes = 8;

struct Level {
    bool defined = false;
    int dim = 2;
    int m = 0;          // nodes per side
    int n = 0, ne = 0;  // nodes, elements
    double h = 0.0, dt = 0.0;
    int nsteps = 0;
    int K = 0;
    double *d_phi = nullptr;         // ne x K
    float *d_phi_hi = nullptr;       // ne x Kp, TF32 high part (tensor-core synthesis)
    float *d_phi_lo = nullptr;       // ne x Kp, remainder
    int Kp = 0;                      // K rounded up to 8
    double *d_theta_mean = nullptr;  // ne or null
    double *d_v0 = nullptr, *d_w0 = nullptr;
    double radius = 0.1;
    mlq::FastDiv divm{};
    int tuned_cs = 0, tuned_npt = 0, tuned_threads = 0;  // set by mlq_autotune (mixed path)
    bool tuned_mg = false;
    // dim 3: mx x my x mz nodes on [0, Lx] x [0, Ly] x [0, Lz], six Kuhn
    // tetrahedra per cube; the level's FP64 mass stencil and lumped mass
    mlq::Grid3 g3{};
    double Lx = 1.0, Ly = 1.0, Lz = 0.25;
    double *d_M3 = nullptr, *d_lump = nullptr;
    // general simplicial level (mlq_add_level_mesh): the tetrahedral mesh and
    // its solver, and the node coordinates for the initial disk
    mlq_mesh *mesh = nullptr;
    std::vector<double> xyz_h;
    std::vector<int32_t> conn_h;   // ne x 4, for point location
    // point QoIs (mlq_set_points): simplex nodes and barycentric weights
    int npts = 0;
    double u_th = 0.0;
    int *d_pt_node = nullptr;      // [npts][4]
    double *d_pt_w = nullptr;      // [npts][4]
};

struct Member {
    int level = 0;
    int64_t S = 0;
    const double *d_xi = nullptr;
    // workspace pieces
    double *cs2 = nullptr, *A64 = nullptr, *v = nullptr, *w = nullptr, *b = nullptr, *y = nullptr, *q = nullptr;
    void *Ai = nullptr, *r = nullptr, *s = nullptr, *wc = nullptr, *p = nullptr, *x = nullptr, *u = nullptr;
    int32_t *iters = nullptr, *status = nullptr;
    float *mgA[mlq::kMgMaxLevels] = {};    // coarse-level stencils (multigrid)
    mlq::D3 *mgD[mlq::kMgMaxLevels] = {};  // coarse-level mean conductivities
    float *mg3v[mlq::kMg3MaxLevels][4] = {};  // 3D multigrid work vectors xa, xb, rr, bb
    mlq::PointArgs pq{};   // point QoIs of this member (npts = 0: none)
    mlq::MeshWs mws{};     // general-mesh level: the solver's workspace
    unsigned *bar3 = nullptr;   // 3D cooperative shape: per-sample barrier words
    double *part3 = nullptr;    // 3D cooperative shape: per-CTA partial sums
};

// 3D multigrid in use for a level (FP32 inner path)
bool uses_mg3(const mlq_ctx *ctx, const Level &L);

// entries per sample of a level's device arrays (3D: rows padded, Grid3)
inline int64_t stored(const Level &L) { return L.dim == 3 ? (int64_t)L.g3.n : (int64_t)L.n; }

// the initial disk v = 1 where |x|^2 <= radius^2 (every coordinate of the
// node), w = 0, of a general level, uploaded to d_v0
int upload_mesh_disk(Level &L)
{
    const int64_t n = (int64_t)L.xyz_h.size() / 3;
    std::vector<double> v0((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const double *x = &L.xyz_h[(size_t)i * 3];
        v0[(size_t)i] = (x[0] * x[0] + x[1] * x[1] + x[2] * x[2] <= L.radius * L.radius) ? 1.0 : 0.0;
    }
    cudaFree(L.d_w0);
    L.d_w0 = nullptr;
    if (!L.d_v0 && cudaMalloc(&L.d_v0, sizeof(double) * (size_t)n) != cudaSuccess) return MLQ_ECUDA;
    if (cudaMemcpy(L.d_v0, v0.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
        return MLQ_ECUDA;
    return MLQ_OK;
}

// free a level's device arrays and its general mesh; the level is undefined after
void release_level(Level &L)
{
    cudaFree(L.d_phi);
    cudaFree(L.d_phi_hi);
    cudaFree(L.d_phi_lo);
    cudaFree(L.d_theta_mean);
    cudaFree(L.d_v0);
    cudaFree(L.d_w0);
    cudaFree(L.d_M3);
    cudaFree(L.d_lump);
    cudaFree(L.d_pt_node);
    cudaFree(L.d_pt_w);
    if (L.mesh) mlq_mesh_destroy(L.mesh);
    L = Level();
}

// multigrid levels below the fine one: m_c = (m_{c-1} + 1) / 2 while m_c >= 3
int mg_coarse_levels(int m)
{
    int c = 0;
    while (c + 1 < mlq::kMgMaxLevels && m >= 5 && (m - 1) % 2 == 0) {
        m = (m + 1) / 2;
        ++c;
    }
    return c;
}

}  // namespace

struct Server;  // request queue and worker of mlq_submit / mlq_poll

// takes the context's lock for the rest of the calling scope (ctx may be null)
#define MLQ_GUARD(c)                                      \
    std::unique_lock<std::recursive_mutex> mlq_guard_;    \
    if (c) mlq_guard_ = std::unique_lock<std::recursive_mutex>((c)->mu)

struct mlq_ctx {
    // held by every call that uses the device or the level table, and by the
    // serving worker around each batch
    std::recursive_mutex mu;
    // serving worker, created by the first mlq_submit (under mu) and read by
    // mlq_poll without it
    std::atomic<Server *> server{nullptr};
    mlq_scheme scheme{};       // time scheme and ionic model (mlq_set_scheme); ionic 0 = FHN
    int serve_lanes = 4;       // mlq_serve_limits (4 measured best of 1, 2, 4, 6 on the 50/s stream)
    size_t serve_budget = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    mlq_options opt{};
    mlq_model model{};
    Level levels[kMaxLevels];
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t pool[kStreams] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_start = nullptr;  // start of the last solve / estimate (profiling)
    cudaEvent_t ev_join[kStreams] = {};
    int64_t launches = 0;
    int *d_err = nullptr;   // set by kernels whose bounded waits time out
    double *h_sums = nullptr;  // pinned host copy of the per-level sums
    // CUDA graph of the last estimate (options.graphs): replayed while the
    // key (configuration generation, sizes, pointers) is unchanged
    uint64_t generation = 1;
    std::vector<uint64_t> graph_key;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0;
    bool capturing = false;
    std::string cuda_error;
    int max_cluster = 8;
    int occ3d[2][32];   // resident clusters of the 3D solver by precision and cluster size (-1: not asked)
    int64_t res3d[2] = {-1, -1};   // resident CTAs of the 3D solver (256 threads) by precision
    int smem_optin = 48 * 1024;
    int num_sms = 1;
    // optional per-member timing of the slab kernel (CUDA events on the
    // member's stream) and iteration totals of the last solve/estimate
    bool profile = false;
    cudaEvent_t ev_t0[kStreams] = {}, ev_t1[kStreams] = {};
    int nmembers = 0;
    int prof_level[kStreams] = {}, prof_coarse[kStreams] = {}, prof_cs[kStreams] = {}, prof_resident[kStreams] = {};
    int prof_threads[kStreams] = {}, prof_npt[kStreams] = {};
    int64_t prof_samples[kStreams] = {}, prof_nodes[kStreams] = {}, prof_steps[kStreams] = {};
    const int32_t *prof_iters_dev[kStreams] = {};
};

namespace {

#define MLQ_CUDA(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            (ctx)->cuda_error = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return e_ == cudaErrorMemoryAllocation ? MLQ_ENOMEM : MLQ_ECUDA;                 \
        }                                                                                    \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool fastdiv_make(uint32_t d, uint32_t nmax, mlq::FastDiv *out)
{
    // mul = ceil(2^40 / d); exact for n * d < 2^40.  Verify on the range.
    if (d == 0) return false;
    if ((uint64_t)nmax * d >= (1ull << 40)) return false;
    out->d = d;
    out->mul = ((1ull << 40) + d - 1) / d;
    for (uint32_t t = 0; t < nmax; ++t)
        if (out->div(t) != t / d) return false;
    return true;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Launch shape of a level: cluster size, threads per CTA, and where the
// sample's PCG vectors live.
struct Shape {
    int cs, threads;
    bool resident;
    size_t smem;
    int npt;  // > 0: register-resident mixed kernel with this many nodes per thread
    bool mg = false;  // register kernel with the multigrid preconditioner
};

// nodes-per-thread variants compiled for the register-resident kernel
constexpr int kNpt[] = {4, 8, 12, 17};
inline int npt_max_threads(int npt) { return npt >= 12 ? (npt >= 16 ? 512 : 384) : 512; }

int max_active_clusters_reg(mlq_ctx *ctx, int cs, int npt, int threads, size_t smem);

// Register-kernel candidates of a level: for each cluster size whose shared
// layout fits, the smallest nodes-per-thread variant that covers a CTA's rows.
std::vector<Shape> reg_candidates(const mlq_ctx *ctx, const Level &L)
{
    std::vector<Shape> out;
    const int limit = ctx->smem_optin - 2048;
    for (int c = 1; c <= ctx->max_cluster; c *= 2) {
        if (c > L.m) break;
        const mlq::RegPlan rp = mlq::reg_plan(L.m, c);
        if (rp.total > limit) continue;
        for (int npt : kNpt) {
            int th = ((rp.nmax + npt - 1) / npt + 31) / 32 * 32;
            if (th < 32) th = 32;
            if (th > npt_max_threads(npt)) continue;
            out.push_back(Shape{c, th, true, (size_t)rp.total, npt});
            break;
        }
    }
    return out;
}

// Multigrid candidates: every cluster size whose multigrid layout fits.
std::vector<Shape> mg_candidates(const mlq_ctx *ctx, const Level &L)
{
    std::vector<Shape> out;
    const int limit = ctx->smem_optin - 3072;  // room for the static reduction buffers
    for (int c = 1; c <= ctx->max_cluster; c *= 2) {
        if (c > L.m) break;
        const mlq::MgPlan mp = mlq::mg_plan(L.m, c);
        if (mp.nl == 0 || mp.total > limit) continue;
        const int nmax = mp.lv[0].rows_max * L.m;
        for (int npt : {4, 8, 12}) {
            int th = ((nmax + npt - 1) / npt + 31) / 32 * 32;
            if (th < 32) th = 32;
            if (th > npt_max_threads(npt)) continue;
            Shape sh{c, th, true, (size_t)mp.total, npt};
            sh.mg = true;
            out.push_back(sh);
            break;
        }
    }
    return out;
}

// 3D: one sample per group of CS CTAs (256 threads), vectors in global
// memory (bandwidth-bound); a CTA owns my / CS grid lines of every plane (a
// CTA may own none).  When the resident CTAs over the samples exceed 16
// (and keep >= 4096 nodes each), that many CTAs per sample in one
// cooperative launch (every SM holds the same CTAs; cs > 16 below).  Else the
// largest cluster size whose clusters hold every
// sample of the batch at once, keeping >= 4096 nodes per CTA; when no
// size holds them all (the batch fills the GPU in any case), one CTA per
// sample.  Clusters of 16 occupy 8 x 16 = 128 of the 152 SMs, 12 and 6
// pack the GPCs more densely.
int active_3d(mlq_ctx *ctx, bool f32, int cs, int threads)
{
    if (cs > 16) return f32 ? mlq::active_3d_f32(cs, threads) : mlq::active_3d_f64(cs, threads);
    int &c = ctx->occ3d[f32 ? 0 : 1][cs & 31];
    if (threads == 256 && c >= 0) return c;
    const int a = f32 ? mlq::active_3d_f32(cs, threads) : mlq::active_3d_f64(cs, threads);
    if (threads == 256) c = a;
    return a;
}

Shape choose_launch_3d(mlq_ctx *ctx, const Level &L, int64_t S = 0)
{
    static const int kCs[] = {16, 12, 8, 6, 4, 2, 1};
    const bool f32 = ctx->opt.precision == MLQ_MIXED;
    int threads = ctx->opt.threads > 0 ? ctx->opt.threads / 32 * 32 : 256;
    threads = std::min(256, std::max(32, threads));
    int cs = 1;
    const int64_t Sx = std::max<int64_t>(S, 1);
    int64_t resident;
    if (threads == 256) {
        int64_t &res = ctx->res3d[f32 ? 0 : 1];   // cached for the default block size
        if (res < 0) res = f32 ? mlq::resident_3d_f32(threads) : mlq::resident_3d_f64(threads);
        resident = res;
    } else {
        resident = f32 ? mlq::resident_3d_f32(threads) : mlq::resident_3d_f64(threads);
    }
    const int64_t G = resident / Sx;
    if (ctx->opt.cluster > 16) {
        cs = ctx->opt.cluster;   // that many CTAs per sample, cooperative launch
    } else if (ctx->opt.cluster > 0) {
        // the built size at or below the requested one that fits the level
        for (int c : kCs)
            if (c <= ctx->opt.cluster && c <= ctx->max_cluster) {
                cs = c;
                break;
            }
    } else if (G > 16 && L.n / G >= 4096) {
        // clusters cannot give every SM the same share: spread each sample
        // over the resident CTAs in one cooperative launch
        cs = (int)G;
    } else {
        for (int c : kCs) {
            if (c > 1 && (c > ctx->max_cluster || L.n / c < 4096)) continue;
            if (active_3d(ctx, f32, c, threads) >= std::max<int64_t>(S, 1)) {
                cs = c;
                break;
            }
        }
    }
    return Shape{cs, threads, false, 0, 0};
}

bool uses_mg3(const mlq_ctx *ctx, const Level &L)
{
    if (L.dim != 3 || ctx->opt.precision != MLQ_MIXED || ctx->opt.precond != 1) return false;
    mlq::Grid3 gl[mlq::kMg3MaxLevels];
    return mlq::mg3_hierarchy(L.g3, gl, mlq::kMg3MaxLevels) > 1;
}

Shape choose_launch(mlq_ctx *ctx, const Level &L, int64_t S = 0)
{
    if (L.mesh) {
        // CTAs per sample: a cluster, or G CTAs of a cooperative launch
        const mlq::MeshShape m = mlq::mesh_member_shape(L.mesh, std::max<int64_t>(S, 1), ctx->opt.cluster);
        return Shape{m.G > 0 ? m.G : m.cs, 512, false, 0, 0};
    }
    if (L.dim == 3) return choose_launch_3d(ctx, L, S);
    // 2D kernels are built for clusters of 1, 2, 4, 8, 16: a request of 6 or
    // 12 takes the power of two below it
    const int creq = ctx->opt.cluster == 6 ? 4 : ctx->opt.cluster == 12 ? 8 : std::min(ctx->opt.cluster, 16);
    const bool paper = ctx->scheme.ionic == 1;   // the paper's scheme runs in the generic slab kernel
    if (!paper && ctx->opt.precision == MLQ_MIXED && ctx->opt.precond == 1 && ctx->opt.storage != 2) {
        if (L.tuned_cs > 0 && L.tuned_mg && creq <= 0 && ctx->opt.threads <= 0) {
            Shape sh{L.tuned_cs, L.tuned_threads, true, (size_t)mlq::mg_plan(L.m, L.tuned_cs).total, L.tuned_npt};
            sh.mg = true;
            return sh;
        }
        std::vector<Shape> cand = mg_candidates(ctx, L);
        for (const Shape &c : cand)
            if (creq <= 0 || c.cs == creq) return c;
    }
    if (L.tuned_mg && ctx->opt.precond != 1) {
        // a multigrid tuning does not apply to the Jacobi kernel
    }
    const int ti = ctx->opt.precision == MLQ_MIXED ? 4 : 8;
    const int limit = ctx->smem_optin - 2048;  // room for the static reduction buffers
    const bool allow = ctx->opt.storage != 2;
    // mixed path: the register-resident kernel when a shape fits
    if (ti == 4 && allow && !paper) {
        if (L.tuned_cs > 0 && !L.tuned_mg && creq <= 0 && ctx->opt.threads <= 0) {
            const mlq::RegPlan rp = mlq::reg_plan(L.m, L.tuned_cs);
            return Shape{L.tuned_cs, L.tuned_threads, true, (size_t)rp.total, L.tuned_npt};
        }
        std::vector<Shape> cand = reg_candidates(ctx, L);
        if (creq > 0 || ctx->opt.threads > 0) {
            // honour explicit overrides when a register shape matches them
            for (const Shape &c : cand) {
                if (creq > 0 && c.cs != creq) continue;
                Shape sh = c;
                if (ctx->opt.threads > 0) {
                    const mlq::RegPlan rp = mlq::reg_plan(L.m, c.cs);
                    bool ok = false;
                    for (int npt : kNpt)
                        if ((int64_t)ctx->opt.threads * npt >= rp.nmax && ctx->opt.threads <= npt_max_threads(npt)) {
                            sh.npt = npt;
                            sh.threads = ctx->opt.threads;
                            ok = true;
                            break;
                        }
                    if (!ok) continue;
                }
                return sh;
            }
        } else if (!cand.empty()) {
            // cost model: waves of co-resident clusters x per-iteration time,
            // t_iter ~ 0.8 us + 0.3 us log2(cluster) + 0.3 ns per node of a CTA
            double best = 1e300;
            Shape pick = cand[0];
            for (const Shape &c : cand) {
                const int act = max_active_clusters_reg(ctx, c.cs, c.npt, c.threads, c.smem);
                if (act <= 0) continue;
                const double waves = S > 0 ? (double)((S + act - 1) / act) : 1.0;
                const int nodes = mlq::reg_plan(L.m, c.cs).nmax;
                const double t = waves * (0.8 + 0.3 * std::log2((double)c.cs) + 3e-4 * nodes);
                if (t < best) {
                    best = t;
                    pick = c;
                }
            }
            return pick;
        }
    }
    Shape sh{0, 0, false, 0, 0};
    auto fits = [&](int c) {
        if (c > L.m) return false;
        return mlq::smem_plan(L.m, c, ti, true).total <= limit;
    };
    if (creq > 0) {
        sh.cs = creq;
        sh.resident = allow && fits(sh.cs);
    } else {
        for (int c = 1; allow && c <= ctx->max_cluster; c *= 2) {
            if (fits(c) && (L.n + c - 1) / c <= 4608) {
                sh.cs = c;
                sh.resident = true;
                break;
            }
        }
        if (!sh.resident) {
            int c = 1;
            while (c < ctx->max_cluster && (L.n + c - 1) / c > 4096) c *= 2;
            sh.cs = c;
        }
    }
    int t = ctx->opt.threads;
    if (t <= 0) {
        const int per = (L.n + sh.cs - 1) / sh.cs;
        t = per >= 2048 ? 512 : (per >= 768 ? 256 : 128);
    }
    sh.threads = t;
    sh.smem = (size_t)mlq::smem_plan(L.m, sh.cs, ti, sh.resident).total;
    return sh;
}

cudaError_t launch_reg_any(int cs, int npt, const mlq::SolveArgs<float> &a, int ncl, int threads, size_t smem,
                           cudaStream_t st)
{
    switch (cs) {
    case 1: return mlq::launch_reg_cs1(npt, a, ncl, threads, smem, st);
    case 2: return mlq::launch_reg_cs2(npt, a, ncl, threads, smem, st);
    case 4: return mlq::launch_reg_cs4(npt, a, ncl, threads, smem, st);
    case 8: return mlq::launch_reg_cs8(npt, a, ncl, threads, smem, st);
    case 16: return mlq::launch_reg_cs16(npt, a, ncl, threads, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mg_any(int cs, int npt, const mlq::SolveArgs<float> &a, const mlq::MgPtrs &ptrs,
                          const mlq::MgPlan &plan, int ncl, int threads, cudaStream_t st)
{
    switch (cs) {
    case 1: return mlq::launch_mg_cs1(npt, a, ptrs, plan, ncl, threads, st);
    case 2: return mlq::launch_mg_cs2(npt, a, ptrs, plan, ncl, threads, st);
    case 4: return mlq::launch_mg_cs4(npt, a, ptrs, plan, ncl, threads, st);
    case 8: return mlq::launch_mg_cs8(npt, a, ptrs, plan, ncl, threads, st);
    case 16: return mlq::launch_mg_cs16(npt, a, ptrs, plan, ncl, threads, st);
    default: return cudaErrorInvalidValue;
    }
}

int max_active_clusters_reg(mlq_ctx *ctx, int cs, int npt, int threads, size_t smem)
{
    (void)ctx;
    switch (cs) {
    case 1: return mlq::active_reg_cs1(npt, threads, smem);
    case 2: return mlq::active_reg_cs2(npt, threads, smem);
    case 4: return mlq::active_reg_cs4(npt, threads, smem);
    case 8: return mlq::active_reg_cs8(npt, threads, smem);
    case 16: return mlq::active_reg_cs16(npt, threads, smem);
    default: return 0;
    }
}

template <typename TI>
cudaError_t launch_slab_cs(int cs, const mlq::SolveArgs<TI> &a, int nclusters, int threads, size_t smem,
                           bool resident, cudaStream_t st)
{
    if constexpr (sizeof(TI) == 4) return mlq::launch_slab_f32(cs, resident, a, nclusters, threads, smem, st);
    else return mlq::launch_slab_f64(cs, resident, a, nclusters, threads, smem, st);
}

// Bytes of workspace for one member (level, S samples).
size_t member_bytes(const mlq_ctx *ctx, const Level &L, int64_t S)
{
    const bool mixed = ctx->opt.precision == MLQ_MIXED;
    if (L.mesh) return mlq::mesh_member_bytes(L.mesh, mixed, S, mlq::mesh_member_shape(L.mesh, S, ctx->opt.cluster));
    const size_t ti = mixed ? 4 : 8;
    const size_t sn = (size_t)S * stored(L);
    size_t t = 0;
    auto add = [&](size_t bytes) { t += align_up(bytes, 256); };
    if (L.dim == 3) {
        add((size_t)S * L.ne * 2 * 8);                 // cs2
        add(sn * mlq::kSlots3D * 8);                    // A64
        if (mixed) add(sn * mlq::kSlots3D * 4);         // A32
        add(mlq::kVRing * sn * 8);                      // v (last solutions and guess)
        add(2 * sn * 8);                                // w
        add(sn * 8);                                    // b
        add(sn * 8);                                    // y
        for (int k = 0; k < 6; ++k) add(sn * ti);       // r u w s p x
        add((size_t)S * 8);
        add((size_t)S * 4);
        add((size_t)S * 4);
        const int cs3 = choose_launch_3d(const_cast<mlq_ctx *>(ctx), L, S).cs;
        if (cs3 > 16) {
            add((size_t)S * 2 * sizeof(unsigned));
            add((size_t)S * 2 * cs3 * 4 * 8);
        }
        if (uses_mg3(ctx, L)) {
            mlq::Grid3 gl[mlq::kMg3MaxLevels];
            const int nl = mlq::mg3_hierarchy(L.g3, gl, mlq::kMg3MaxLevels);
            add(sn * 4);                                // level-0 xa
            add(sn * 4);                                // level-0 xb
            for (int c = 1; c < nl; ++c) {
                const size_t nc = (size_t)S * gl[c].n;
                const size_t nec = (size_t)S * 6 * (gl[c].mx - 1) * (gl[c].my - 1) * (gl[c].mz - 1);
                add(nec * 3 * 4);                       // mean D
                add(nc * mlq::kSlots3D * 4);            // stencil
                for (int k = 0; k < 4; ++k) add(nc * 4);
            }
        }
        return t;
    }
    add((size_t)S * L.ne * 2 * 8);          // cs2
    add(sn * mlq::kSlots2D * 8);            // A64
    if (mixed) add(sn * mlq::kSlots2D * 4); // A32
    add((mixed && ctx->opt.precond == 1 ? mlq::kVRing : 1) * sn * 8);  // v (multigrid: last solutions and guess)
    add(2 * sn * 8);                        // w
    add(sn * 8);                            // b
    if (mixed && ctx->opt.precond == 1) add(sn * 8);  // y (multigrid kernel)
    add(2 * sn * ti);                       // r
    add(2 * sn * ti);                       // s
    add(2 * sn * ti);                       // wc
    add(sn * ti);                           // p
    add(sn * ti);                           // x
    add((size_t)S * 8);                     // q
    add((size_t)S * 4);                     // iters
    add((size_t)S * 4);                     // status
    if (mixed && ctx->opt.precond == 1) {
        int mc = L.m;
        for (int c = 1; c <= mg_coarse_levels(L.m); ++c) {
            mc = (mc + 1) / 2;
            add((size_t)S * mlq::kSlots2D * mc * mc * 4);
            add((size_t)S * 2 * (mc - 1) * (mc - 1) * sizeof(mlq::D3));
        }
    }
    return t;
}

void member_carve(const mlq_ctx *ctx, const Level &L, Member &mb, char *&cur)
{
    const bool mixed = ctx->opt.precision == MLQ_MIXED;
    if (L.mesh) {
        mb.mws = mlq::mesh_member_carve(L.mesh, mixed, mb.S, mlq::mesh_member_shape(L.mesh, mb.S, ctx->opt.cluster), cur);
        mb.q = mb.mws.q;
        mb.iters = mb.mws.iters;
        mb.status = mb.mws.status;
        return;
    }
    const size_t ti = mixed ? 4 : 8;
    const size_t sn = (size_t)mb.S * stored(L);
    auto take = [&](size_t bytes) {
        char *p = cur;
        cur += align_up(bytes, 256);
        return (void *)p;
    };
    if (L.dim == 3) {
        mb.cs2 = (double *)take((size_t)mb.S * L.ne * 2 * 8);
        mb.A64 = (double *)take(sn * mlq::kSlots3D * 8);
        mb.Ai = mixed ? take(sn * mlq::kSlots3D * 4) : (void *)mb.A64;
        mb.v = (double *)take(mlq::kVRing * sn * 8);
        mb.w = (double *)take(2 * sn * 8);
        mb.b = (double *)take(sn * 8);
        mb.y = (double *)take(sn * 8);
        mb.r = take(sn * ti);
        mb.u = take(sn * ti);
        mb.wc = take(sn * ti);
        mb.s = take(sn * ti);
        mb.p = take(sn * ti);
        mb.x = take(sn * ti);
        mb.q = (double *)take((size_t)mb.S * 8);
        mb.iters = (int32_t *)take((size_t)mb.S * 4);
        mb.status = (int32_t *)take((size_t)mb.S * 4);
        const int cs3 = choose_launch_3d(const_cast<mlq_ctx *>(ctx), L, mb.S).cs;
        if (cs3 > 16) {
            mb.bar3 = (unsigned *)take((size_t)mb.S * 2 * sizeof(unsigned));
            mb.part3 = (double *)take((size_t)mb.S * 2 * cs3 * 4 * 8);
        }
        if (uses_mg3(ctx, L)) {
            mlq::Grid3 gl[mlq::kMg3MaxLevels];
            const int nl = mlq::mg3_hierarchy(L.g3, gl, mlq::kMg3MaxLevels);
            mb.mg3v[0][0] = (float *)take(sn * 4);
            mb.mg3v[0][1] = (float *)take(sn * 4);
            for (int c = 1; c < nl; ++c) {
                const size_t nc = (size_t)mb.S * gl[c].n;
                const size_t nec = (size_t)mb.S * 6 * (gl[c].mx - 1) * (gl[c].my - 1) * (gl[c].mz - 1);
                mb.mgD[c] = (mlq::D3 *)take(nec * 3 * 4);
                mb.mgA[c] = (float *)take(nc * mlq::kSlots3D * 4);
                for (int k = 0; k < 4; ++k) mb.mg3v[c][k] = (float *)take(nc * 4);
            }
        }
        return;
    }
    mb.cs2 = (double *)take((size_t)mb.S * L.ne * 2 * 8);
    mb.A64 = (double *)take(sn * mlq::kSlots2D * 8);
    mb.Ai = mixed ? take(sn * mlq::kSlots2D * 4) : (void *)mb.A64;
    mb.v = (double *)take((mixed && ctx->opt.precond == 1 ? mlq::kVRing : 1) * sn * 8);
    mb.w = (double *)take(2 * sn * 8);
    mb.b = (double *)take(sn * 8);
    mb.y = (mixed && ctx->opt.precond == 1) ? (double *)take(sn * 8) : nullptr;
    mb.r = take(2 * sn * ti);
    mb.s = take(2 * sn * ti);
    mb.wc = take(2 * sn * ti);
    mb.p = take(sn * ti);
    mb.x = take(sn * ti);
    mb.q = (double *)take((size_t)mb.S * 8);
    mb.iters = (int32_t *)take((size_t)mb.S * 4);
    mb.status = (int32_t *)take((size_t)mb.S * 4);
    if (mixed && ctx->opt.precond == 1) {
        int mc = L.m;
        for (int c = 1; c <= mg_coarse_levels(L.m); ++c) {
            mc = (mc + 1) / 2;
            mb.mgA[c] = (float *)take((size_t)mb.S * mlq::kSlots2D * mc * mc * 4);
            mb.mgD[c] = (mlq::D3 *)take((size_t)mb.S * 2 * (mc - 1) * (mc - 1) * sizeof(mlq::D3));
        }
    }
}

int ensure_workspace(mlq_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return MLQ_OK;
    if (ctx->ws) {
        MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        MLQ_CUDA(ctx, cudaFree(ctx->ws));
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    MLQ_CUDA(ctx, cudaMalloc(&ctx->ws, bytes));
    ctx->ws_bytes = bytes;
    return MLQ_OK;
}

// the carve of a call stays inside the workspace it sized (a piece past the
// end would be taken for host memory by the copy engine)
int carve_check(mlq_ctx *ctx, const char *cur, size_t more)
{
    if ((size_t)(cur - (const char *)ctx->ws) + more > ctx->ws_bytes) {
        ctx->cuda_error = "internal: workspace carve exceeds the sized workspace";
        return MLQ_ENOMEM;
    }
    return MLQ_OK;
}

// K1.  Mixed path: tensor cores (TF32 split, FP32-accurate); FP64 path: FP64
// on the CUDA cores (the 1e-10 parity of that path needs the FP64 angle).
int launch_synthesis(mlq_ctx *ctx, const Level &L, const double *d_xi, int S, double *cs2, cudaStream_t st)
{
    if (ctx->opt.precision == MLQ_MIXED && L.d_phi_hi) {
        const size_t limit = 200 * 1024;
        int NT = ((S + 15) / 16) * 16;
        if (NT > 256) NT = 256;
        while (NT > 16 && (size_t)2 * (mlq::kTcM + NT) * L.Kp * 4 + 64 > limit) NT -= 16;
        const size_t smem = (size_t)2 * (mlq::kTcM + NT) * L.Kp * 4 + 64;
        if (smem <= limit) {
            MLQ_CUDA(ctx, cudaFuncSetAttribute(mlq::kl_synthesis_tc_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            dim3 grd((unsigned)((L.ne + mlq::kTcM - 1) / mlq::kTcM), (unsigned)((S + NT - 1) / NT));
            mlq::kl_synthesis_tc_kernel<<<grd, 128, smem, st>>>(L.d_phi_hi, L.d_phi_lo, L.d_theta_mean, d_xi, L.K,
                                                                 L.Kp, L.ne, S, NT, cs2, ctx->d_err);
            MLQ_CUDA(ctx, cudaGetLastError());
            ctx->launches++;
            return MLQ_OK;
        }
    }
    dim3 blk(256), grd((unsigned)((L.ne + 255) / 256), (unsigned)S);
    mlq::kl_synthesis_kernel<<<grd, blk, 0, st>>>(L.d_phi, L.d_theta_mean, d_xi, L.K, L.ne, S, cs2);
    MLQ_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    return MLQ_OK;
}

// Member launch phases: set-up (KL synthesis, stencils, multigrid levels)
// and the slab solve; an estimate runs every member's set-up before the first
// solve so that the long solver kernels do not hold SMs the set-ups wait for.
enum { kSetup = 1, kSolve = 2, kBoth = 3 };

// 3D member: K1 as in 2D, the 15-point stencil set-up, the global-memory
// cluster solver
template <typename TI>
int launch_member3d_t(mlq_ctx *ctx, const Level &L, const Member &mb, cudaStream_t st, int slot, int phase)
{
    const bool mixed = sizeof(TI) == 4;
    if (phase & kSetup) {
        int st1 = launch_synthesis(ctx, L, mb.d_xi, (int)mb.S, mb.cs2, st);
        if (st1 != MLQ_OK) return st1;
        MLQ_CUDA(ctx, mlq::launch_stencil3d_setup(mb.cs2, L.g3, L.dt, ctx->model.s_l, ctx->model.s_t, (int)mb.S,
                                                  mb.A64, mixed ? (float *)mb.Ai : nullptr, st));
        ctx->launches++;
        if (uses_mg3(ctx, L)) {
            mlq::Grid3 gl[mlq::kMg3MaxLevels];
            const int nl = mlq::mg3_hierarchy(L.g3, gl, mlq::kMg3MaxLevels);
            for (int c = 1; c < nl; ++c) {
                MLQ_CUDA(ctx, mlq::launch_mg3_setup(c == 1 ? mb.cs2 : nullptr, c == 1 ? nullptr : (const float *)mb.mgD[c - 1],
                                                    gl[c - 1], gl[c], (int)mb.S, L.dt, ctx->model.s_l,
                                                    ctx->model.s_t, (float *)mb.mgD[c], mb.mgA[c], st));
                ctx->launches += 2;
            }
        }
    }
    if (!(phase & kSolve)) return MLQ_OK;
    mlq::Solve3Args<TI> a{};
    a.g = L.g3;
    a.Lx = L.Lx;
    a.Ly = L.Ly;
    a.Lz = L.Lz;
    a.dt = L.dt;
    a.nsteps = L.nsteps;
    a.a = ctx->model.a;
    a.eps = ctx->model.eps;
    a.gam = ctx->model.gamma;
    a.rtol_out = ctx->opt.rtol;
    a.rtol_in = ctx->opt.rtol_inner;
    a.max_iter = ctx->opt.max_iter;
    a.max_sweeps = mixed ? ctx->opt.max_sweeps : 1;
    a.M3 = L.d_M3;
    a.lump = L.d_lump;
    a.A64 = mb.A64;
    a.Ai = (const TI *)mb.Ai;
    a.v = mb.v;
    a.w = mb.w;
    a.b = mb.b;
    a.y = mb.y;
    a.r = (TI *)mb.r;
    a.u = (TI *)mb.u;
    a.wv = (TI *)mb.wc;
    a.s = (TI *)mb.s;
    a.p = (TI *)mb.p;
    a.x = (TI *)mb.x;
    a.v0 = L.d_v0;
    a.w0 = L.d_w0;
    a.radius2 = L.radius * L.radius;
    a.S = (int)mb.S;
    a.q = mb.q;
    a.iters = mb.iters;
    a.status = mb.status;
    a.pq = mb.pq;
    a.mg.nl = 1;
    if (uses_mg3(ctx, L)) {
        a.mg.nl = mlq::mg3_hierarchy(L.g3, a.mg.g, mlq::kMg3MaxLevels);
        a.mg.omega = 0.7f;  // lambda_max(D^-1 A) <= 2.4 for P1 on Kuhn tetrahedra
        a.mg.xa[0] = mb.mg3v[0][0];
        a.mg.xb[0] = mb.mg3v[0][1];
        for (int c = 1; c < a.mg.nl; ++c) {
            a.mg.A[c] = mb.mgA[c];
            a.mg.xa[c] = mb.mg3v[c][0];
            a.mg.xb[c] = mb.mg3v[c][1];
            a.mg.rr[c] = mb.mg3v[c][2];
            a.mg.bb[c] = mb.mg3v[c][3];
        }
    }
    const Shape sh = choose_launch_3d(ctx, L, mb.S);
    const bool timed = ctx->profile && slot >= 0 && slot < kStreams;
    const unsigned evf = ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (timed) MLQ_CUDA(ctx, cudaEventRecordWithFlags(ctx->ev_t0[slot], st, evf));
    if (sh.cs > 16 && active_3d(ctx, sizeof(TI) == 4, sh.cs, sh.threads) < mb.S) return MLQ_EUNSUPPORTED;
    if constexpr (sizeof(TI) == 4)
        MLQ_CUDA(ctx, mlq::launch_3d_f32(sh.cs, a, (int)mb.S, sh.threads, st, mb.bar3, mb.part3, ctx->d_err));
    else MLQ_CUDA(ctx, mlq::launch_3d_f64(sh.cs, a, (int)mb.S, sh.threads, st, mb.bar3, mb.part3, ctx->d_err));
    if (timed) MLQ_CUDA(ctx, cudaEventRecordWithFlags(ctx->ev_t1[slot], st, evf));
    ctx->launches++;
    return MLQ_OK;
}

// general-mesh member: KL synthesis and CSR assembly, then the block loop
// of the general-mesh solver (Jacobi-PCG, FP64 or FP32 inside FP64
// refinement by the context's precision)
int launch_member_mesh(mlq_ctx *ctx, const Level &L, const Member &mb, cudaStream_t st, int slot, int phase)
{
    const mlq::MeshShape sh = mlq::mesh_member_shape(L.mesh, mb.S, ctx->opt.cluster);
    if (sh.cs < 1) return MLQ_EUNSUPPORTED;   // the requested CTAs per sample cannot all be resident
    const bool timed = ctx->profile && slot >= 0 && slot < kStreams && (phase & kSolve);
    const unsigned evf = ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (phase & kSetup) {
        MLQ_CUDA(ctx, mlq::mesh_member_launch(L.mesh, ctx->model, ctx->opt, L.dt, L.nsteps, L.d_v0, L.d_w0, mb.S, mb.d_xi,
                                              mb.mws, sh, ctx->d_err, st, true, false));
        ctx->launches += ctx->opt.precision == MLQ_MIXED ? 3 : 2;
    }
    if (!(phase & kSolve)) return MLQ_OK;
    if (timed) MLQ_CUDA(ctx, cudaEventRecordWithFlags(ctx->ev_t0[slot], st, evf));
    MLQ_CUDA(ctx, mlq::mesh_member_launch(L.mesh, ctx->model, ctx->opt, L.dt, L.nsteps, L.d_v0, L.d_w0, mb.S, mb.d_xi,
                                          mb.mws, sh, ctx->d_err, st, false, true, &mb.pq));
    if (timed) MLQ_CUDA(ctx, cudaEventRecordWithFlags(ctx->ev_t1[slot], st, evf));
    ctx->launches++;
    return MLQ_OK;
}

template <typename TI>
int launch_member_t(mlq_ctx *ctx, const Level &L, const Member &mb, cudaStream_t st, int slot, int phase)
{
    if (L.mesh) return launch_member_mesh(ctx, L, mb, st, slot, phase);
    if (L.dim == 3) return launch_member3d_t<TI>(ctx, L, mb, st, slot, phase);
    const bool mixed = sizeof(TI) == 4;
    // K1: KL synthesis (theta -> cos 2t, sin 2t)
    if (phase & kSetup) {
        int st1 = launch_synthesis(ctx, L, mb.d_xi, (int)mb.S, mb.cs2, st);
        if (st1 != MLQ_OK) return st1;
    }
    // K2: stencil of A = M + dt K(theta)
    if (phase & kSetup) {
        dim3 blk(256), grd((unsigned)((L.n + 255) / 256), (unsigned)mb.S);
        // A = M + theta dt K (theta = 1 unless the paper's Crank-Nicolson scheme is set)
        const double dtk = ctx->scheme.ionic == 1 ? ctx->scheme.theta * L.dt : L.dt;
        mlq::stencil_setup_kernel<<<grd, blk, 0, st>>>(mb.cs2, L.m, L.h, dtk, ctx->model.s_l, ctx->model.s_t,
                                                         (int)mb.S, mb.A64, mixed ? (float *)mb.Ai : nullptr);
        MLQ_CUDA(ctx, cudaGetLastError());
        ctx->launches++;
    }
    // K3-K6: all time blocks
    mlq::SolveArgs<TI> a{};
    a.m = L.m;
    a.n = L.n;
    a.divm = L.divm;
    a.h2 = L.h * L.h;
    a.dt = L.dt;
    a.nsteps = L.nsteps;
    a.a = ctx->model.a;
    a.eps = ctx->model.eps;
    a.gam = ctx->model.gamma;
    a.rtol_out = ctx->opt.rtol;
    a.rtol_in = ctx->opt.rtol_inner;
    a.max_iter = ctx->opt.max_iter;
    a.max_sweeps = mixed ? ctx->opt.max_sweeps : 1;
    a.A64 = mb.A64;
    a.Ai = (const TI *)mb.Ai;
    a.v = mb.v;
    a.w = mb.w;
    a.b = mb.b;
    a.y = mb.y;
    a.r = (TI *)mb.r;
    a.s = (TI *)mb.s;
    a.wc = (TI *)mb.wc;
    a.p = (TI *)mb.p;
    a.x = (TI *)mb.x;
    a.v0 = L.d_v0;
    a.w0 = L.d_w0;
    a.radius2 = L.radius * L.radius;
    a.S = (int)mb.S;
    a.q = mb.q;
    a.iters = mb.iters;
    a.status = mb.status;
    a.pq = mb.pq;
    if (ctx->scheme.ionic == 1) {
        const mlq_scheme &sc = ctx->scheme;
        a.scheme = 1;
        a.theta = sc.theta;
        a.alpha = sc.alpha;
        a.u_rest = sc.u_rest;
        a.u_th = sc.u_th;
        a.u_peak = sc.u_peak;
        a.amp = sc.amp;
        a.sigma2 = sc.sigma * sc.sigma;
        a.t1 = sc.t1;
        a.x0 = sc.x0[0];
        a.y0 = sc.x0[1];
        // chord-Newton sweeps in both precisions (the FP64 path too)
        a.max_sweeps = std::max(ctx->opt.max_sweeps, 60);
    } else {
        a.scheme = 0;
        a.theta = 1.0;
    }
    const Shape sh = choose_launch(ctx, L, mb.S);
    if (ctx->opt.storage == 1 && !sh.resident) return MLQ_EUNSUPPORTED;
    const bool timed = ctx->profile && slot >= 0 && slot < kStreams;
    const unsigned evf = ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if constexpr (sizeof(TI) == 4) {
        if (sh.mg) {
            const mlq::MgPlan mp = mlq::mg_plan(L.m, sh.cs);
            mlq::MgPtrs ptrs{};
            int mc = L.m;
            for (int c = 1; c < mp.nl; ++c) {
                const int mf = mc;
                mc = (mc + 1) / 2;
                const int nec = 2 * (mc - 1) * (mc - 1);
                if (phase & kSetup) {
                    mlq::mg_coarsen_kernel<<<dim3((unsigned)((nec + 255) / 256), (unsigned)mb.S), 256, 0, st>>>(
                        c == 1 ? mb.cs2 : nullptr, c == 1 ? nullptr : mb.mgD[c - 1], mf, (int)mb.S,
                        ctx->model.s_l, ctx->model.s_t, mb.mgD[c]);
                    mlq::mg_stencil_kernel<<<dim3((unsigned)((mc * mc + 255) / 256), (unsigned)mb.S), 256, 0,
                                             st>>>(mb.mgD[c], mc, L.dt, (int)mb.S, mb.mgA[c]);
                    MLQ_CUDA(ctx, cudaGetLastError());
                    ctx->launches += 2;
                }
                ptrs.A[c] = mb.mgA[c];
            }
            if (!(phase & kSolve)) return MLQ_OK;
            if (timed) MLQ_CUDA(ctx, cudaEventRecordWithFlags(ctx->ev_t0[slot], st, evf));
            MLQ_CUDA(ctx, launch_mg_any(sh.cs, sh.npt, a, ptrs, mp, (int)mb.S, sh.threads, st));
        } else {
            if (!(phase & kSolve)) return MLQ_OK;
            if (timed) MLQ_CUDA(ctx, cudaEventRecordWithFlags(ctx->ev_t0[slot], st, evf));
            if (sh.npt > 0)
                MLQ_CUDA(ctx, launch_reg_any(sh.cs, sh.npt, a, (int)mb.S, sh.threads, sh.smem, st));
            else
                MLQ_CUDA(ctx, launch_slab_cs<TI>(sh.cs, a, (int)mb.S, sh.threads, sh.smem, sh.resident, st));
        }
    } else {
        if (!(phase & kSolve)) return MLQ_OK;
        if (timed) MLQ_CUDA(ctx, cudaEventRecordWithFlags(ctx->ev_t0[slot], st, evf));
        MLQ_CUDA(ctx, launch_slab_cs<TI>(sh.cs, a, (int)mb.S, sh.threads, sh.smem, sh.resident, st));
    }
    if (timed) MLQ_CUDA(ctx, cudaEventRecordWithFlags(ctx->ev_t1[slot], st, evf));
    ctx->launches++;
    return MLQ_OK;
}

int launch_member(mlq_ctx *ctx, const Member &mb, cudaStream_t st, int slot, int coarse, int phase = kBoth)
{
    const Level &L = ctx->levels[mb.level];
    if (ctx->profile && slot >= 0 && slot < kStreams) {
        const Shape sh = choose_launch(ctx, L, mb.S);
        ctx->prof_level[slot] = mb.level;
        ctx->prof_coarse[slot] = coarse;
        ctx->prof_cs[slot] = sh.cs;
        ctx->prof_resident[slot] = sh.mg ? 3 : (sh.npt > 0 ? 2 : (sh.resident ? 1 : 0));
        ctx->prof_threads[slot] = sh.threads;
        ctx->prof_npt[slot] = sh.npt;
        ctx->prof_samples[slot] = mb.S;
        ctx->prof_nodes[slot] = L.n;
        ctx->prof_steps[slot] = L.nsteps;
        ctx->prof_iters_dev[slot] = mb.iters;
        ctx->nmembers = std::max(ctx->nmembers, slot + 1);
    }
    if (ctx->opt.precision == MLQ_MIXED) return launch_member_t<float>(ctx, L, mb, st, slot, phase);
    return launch_member_t<double>(ctx, L, mb, st, slot, phase);
}

// device error flag (a bounded wait ran out): report once and clear
int check_err(mlq_ctx *ctx)
{
    int h = 0;
    MLQ_CUDA(ctx, cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        MLQ_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
        ctx->cuda_error = "a bounded device wait timed out";
        return MLQ_ETIMEOUT;
    }
    return MLQ_OK;
}

int check_level(const mlq_ctx *ctx, int level)
{
    if (level < 0 || level >= kMaxLevels || !ctx->levels[level].defined) return MLQ_EINVAL;
    const Level &L = ctx->levels[level];
    if (L.mesh ? L.K < 1 : !L.d_phi) return MLQ_EINVAL;
    return MLQ_OK;
}

int copy_out(mlq_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (!dst || bytes == 0) return MLQ_OK;
    MLQ_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return MLQ_OK;
}

}  // namespace

// Profiling bookkeeping of a member whose kernels run from a replayed graph.
void launch_member_profile_only(mlq_ctx *ctx, const Member &mb, int slot, int coarse)
{
    const Level &L = ctx->levels[mb.level];
    const Shape sh = choose_launch(ctx, L, mb.S);
    ctx->prof_level[slot] = mb.level;
    ctx->prof_coarse[slot] = coarse;
    ctx->prof_cs[slot] = sh.cs;
    ctx->prof_resident[slot] = sh.mg ? 3 : (sh.npt > 0 ? 2 : (sh.resident ? 1 : 0));
    ctx->prof_threads[slot] = sh.threads;
    ctx->prof_npt[slot] = sh.npt;
    ctx->prof_samples[slot] = mb.S;
    ctx->prof_nodes[slot] = L.n;
    ctx->prof_steps[slot] = L.nsteps;
    ctx->prof_iters_dev[slot] = mb.iters;
    ctx->nmembers = std::max(ctx->nmembers, slot + 1);
}

// Wait for an estimate and combine the per-level FP64 sums on the host.
bool same_shape(const Shape &a, const Shape &b)
{
    return a.cs == b.cs && a.threads == b.threads && a.resident == b.resident && a.smem == b.smem &&
           a.npt == b.npt && a.mg == b.mg;
}

int finish_estimate(mlq_ctx *ctx, int L, const int64_t *N, double *mean_out, double *var_out, double *rmse_out)
{
    MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int st = check_err(ctx);
    if (st != MLQ_OK) return st;
    double mean = 0.0, mse = 0.0;
    for (int l = 0; l <= L; ++l) {
        const double nl = (double)N[l];
        const double v = ctx->h_sums[2 * l + 1] / (nl - 1.0);
        mean += ctx->h_sums[2 * l] / nl;
        mse += v / nl;
        if (var_out) var_out[l] = v;
    }
    *mean_out = mean;
    if (rmse_out) *rmse_out = std::sqrt(mse);
    return MLQ_OK;
}

namespace {
void serve_stop(mlq_ctx *ctx);  // stops and frees the serving worker (below)

// mlq_synthesize on a general-mesh level: the member's set-up phase (the
// general-mesh solver's FP64 synthesis kernel, then its CSR assembly) on
// the context's stream, and a copy of its (cos 2 theta, sin 2 theta) table
// ([S][n_elem][2] FP64, the layout of the structured levels' output).
int synthesize_mesh(mlq_ctx *ctx, int level, int64_t S, const double *xi, double *cs2_out)
{
    const Level &L = ctx->levels[level];
    size_t need = 0;
    int st = mlq_workspace_bytes(ctx, level, S, 0, &need);
    if (st != MLQ_OK) return st;
    if ((st = ensure_workspace(ctx, need)) != MLQ_OK) return st;
    ctx->nmembers = 0;
    char *cur = (char *)ctx->ws;
    Member mf;
    mf.level = level;
    mf.S = S;
    member_carve(ctx, L, mf, cur);
    cur += align_up((size_t)S * 8, 256) + 256 + align_up((size_t)S * 4, 256);  // as mlq_solve's carve
    const double *d_xi = xi;
    if ((st = carve_check(ctx, cur, is_device_ptr(xi) ? 0 : (size_t)S * L.K * 8)) != MLQ_OK) return st;
    if (!is_device_ptr(xi)) {
        double *dx = (double *)cur;
        MLQ_CUDA(ctx, cudaMemcpyAsync(dx, xi, sizeof(double) * S * L.K, cudaMemcpyHostToDevice, ctx->stream));
        d_xi = dx;
    }
    mf.d_xi = d_xi;
    if ((st = launch_member(ctx, mf, ctx->stream, -1, 0, kSetup)) != MLQ_OK) return st;
    if ((st = copy_out(ctx, cs2_out, mf.mws.cs2, (size_t)S * L.ne * 16, ctx->stream)) != MLQ_OK) return st;
    MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}
}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int mlq_default_options(mlq_options *opt, int precision)
{
    if (!opt || (precision != MLQ_FP64 && precision != MLQ_MIXED)) return MLQ_EINVAL;
    opt->precision = precision;
    opt->rtol = precision == MLQ_FP64 ? 1e-13 : 1e-12;
    opt->rtol_inner = 1e-5;
    opt->max_iter = 100000;
    opt->max_sweeps = 20;
    opt->cluster = 0;
    opt->threads = 0;
    opt->storage = 0;
    opt->graphs = 0;
    opt->precond = precision == MLQ_MIXED ? 1 : 0;
    return MLQ_OK;
}

int mlq_default_model(mlq_model *m)
{
    if (!m) return MLQ_EINVAL;
    m->s_l = 1.0;
    m->s_t = 0.2;
    m->a = 0.1;
    m->eps = 0.01;
    m->gamma = 0.5;
    m->T = 10.0;
    return MLQ_OK;
}

static int validate_options(const mlq_options *o)
{
    if (o->precision != MLQ_FP64 && o->precision != MLQ_MIXED) return MLQ_EINVAL;
    if (!(o->rtol > 0.0) || !(o->rtol_inner > 0.0) || o->max_iter < 0 || o->max_sweeps < 1) return MLQ_EINVAL;
    if (o->cluster != 0 && o->cluster != 1 && o->cluster != 2 && o->cluster != 4 && o->cluster != 6 &&
        o->cluster != 8 && o->cluster != 12 && !(o->cluster >= 16 && o->cluster <= 1024))
        return MLQ_EINVAL;
    if (o->threads != 0 && (o->threads < 64 || o->threads > 512 || o->threads % 32)) return MLQ_EINVAL;
    if (o->storage < 0 || o->storage > 2) return MLQ_EINVAL;
    if (o->precond < 0 || o->precond > 1) return MLQ_EINVAL;
    return MLQ_OK;
}

int mlq_create(mlq_ctx **out, int device, void *cuda_stream, const mlq_options *opt)
{
    if (!out) return MLQ_EINVAL;
    *out = nullptr;
    mlq_options o;
    if (opt) o = *opt;
    else mlq_default_options(&o, MLQ_FP64);
    if (validate_options(&o) != MLQ_OK) return MLQ_EINVAL;
    mlq_ctx *ctx = new (std::nothrow) mlq_ctx();
    if (!ctx) return MLQ_ENOMEM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->opt = o;
    mlq_default_model(&ctx->model);
    auto fail = [&](int code) {
        mlq_destroy(ctx);
        return code;
    };
    if (cudaSetDevice(device) != cudaSuccess) return fail(MLQ_ECUDA);
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) return fail(MLQ_ECUDA);
    for (int k = 0; k < kStreams; ++k) {
        // priority by pair: members (2k, 2k+1) of the k-th largest level
        if (cudaStreamCreateWithPriority(&ctx->pool[k], cudaStreamNonBlocking,
                                         std::min(prio_least, prio_greatest + k / 2)) != cudaSuccess)
            return fail(MLQ_ECUDA);
        if (cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming) != cudaSuccess)
            return fail(MLQ_ECUDA);
    }
    if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess) return fail(MLQ_ECUDA);
    if (cudaEventCreate(&ctx->ev_start) != cudaSuccess) return fail(MLQ_ECUDA);
    for (int k = 0; k < kStreams; ++k)
        if (cudaEventCreate(&ctx->ev_t0[k]) != cudaSuccess || cudaEventCreate(&ctx->ev_t1[k]) != cudaSuccess)
            return fail(MLQ_ECUDA);
    // largest cluster that can be resident with our largest shapes
    int nonportable = 0;
    cudaDeviceGetAttribute(&nonportable, cudaDevAttrClusterLaunch, device);
    cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    ctx->max_cluster = mlq::active_reg_cs16(8, 512, 48 * 1024) > 0 ? 16 : 8;
    for (auto &row : ctx->occ3d)
        for (int &c : row) c = -1;
    cudaGetLastError();
    (void)nonportable;
    if (o.cluster > ctx->max_cluster && o.cluster <= 16) return fail(MLQ_EUNSUPPORTED);   // sizes above 16 are cooperative launches
    if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess)
        return fail(MLQ_ENOMEM);
    if (cudaMallocHost(&ctx->h_sums, sizeof(double) * 2 * kMaxLevels) != cudaSuccess) return fail(MLQ_ENOMEM);
    *out = ctx;
    return MLQ_OK;
}

int mlq_destroy(mlq_ctx *ctx)
{
    if (!ctx) return MLQ_EINVAL;
    serve_stop(ctx);
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (int k = 0; k < kStreams; ++k) {
        if (ctx->pool[k]) {
            cudaStreamSynchronize(ctx->pool[k]);
            cudaStreamDestroy(ctx->pool[k]);
        }
        if (ctx->ev_join[k]) cudaEventDestroy(ctx->ev_join[k]);
        if (ctx->ev_t0[k]) cudaEventDestroy(ctx->ev_t0[k]);
        if (ctx->ev_t1[k]) cudaEventDestroy(ctx->ev_t1[k]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    cudaFree(ctx->d_err);
    if (ctx->h_sums) cudaFreeHost(ctx->h_sums);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    for (auto &L : ctx->levels) release_level(L);
    cudaFree(ctx->ws);
    delete ctx;
    return MLQ_OK;
}

int mlq_set_options(mlq_ctx *ctx, const mlq_options *opt)
{
    MLQ_GUARD(ctx);
    if (!ctx || !opt || validate_options(opt) != MLQ_OK) return MLQ_EINVAL;
    ctx->generation++;
    if (opt->cluster > ctx->max_cluster && opt->cluster <= 16) return MLQ_EUNSUPPORTED;
    ctx->opt = *opt;
    return MLQ_OK;
}

int mlq_default_scheme(mlq_scheme *sc)
{
    if (!sc) return MLQ_EINVAL;
    sc->ionic = 0;
    sc->theta = 1.0;
    sc->alpha = 1.4e-3;
    sc->u_rest = 0.0;
    sc->u_th = 28.0;
    sc->u_peak = 115.0;
    sc->amp = 115.0;
    sc->sigma = 0.1;
    sc->t1 = 0.005;
    sc->x0[0] = sc->x0[1] = sc->x0[2] = 0.0;
    return MLQ_OK;
}

int mlq_set_scheme(mlq_ctx *ctx, const mlq_scheme *sc)
{
    MLQ_GUARD(ctx);
    if (!ctx || !sc || (sc->ionic != 0 && sc->ionic != 1)) return MLQ_EINVAL;
    if (sc->ionic == 1 && !(sc->theta > 0.0 && sc->theta <= 1.0 && std::isfinite(sc->alpha) && sc->sigma > 0.0))
        return MLQ_EINVAL;
    for (const Level &L : ctx->levels)
        if (L.defined && L.dim == 3 && sc->ionic == 1) return MLQ_EUNSUPPORTED;
    ctx->scheme = *sc;
    ctx->generation++;
    return MLQ_OK;
}

int mlq_set_model(mlq_ctx *ctx, const mlq_model *m)
{
    MLQ_GUARD(ctx);
    if (!ctx || !m) return MLQ_EINVAL;
    ctx->generation++;
    if (!(m->s_l > 0.0) || !(m->s_t > 0.0) || !(m->T > 0.0)) return MLQ_EINVAL;
    ctx->model = *m;
    return MLQ_OK;
}

int mlq_add_level(mlq_ctx *ctx, int level, int dim, const int32_t *dims, const double *lengths, double dt,
                  int32_t nsteps)
{
    MLQ_GUARD(ctx);
    if (!ctx || !dims || level < 0 || level >= kMaxLevels) return MLQ_EINVAL;
    if (dim != 2 && dim != 3) return MLQ_EINVAL;
    if (!(dt > 0.0) || nsteps < 0) return MLQ_EINVAL;
    if (dim == 3 && ctx->scheme.ionic == 1) return MLQ_EUNSUPPORTED;   // the paper's scheme is 2D only
    if (dim == 3) {
        const int64_t nn = (int64_t)dims[0] * dims[1] * dims[2];
        // nine stencil slots of a sample must stay within 32-bit indices
        if (dims[0] < 2 || dims[1] < 2 || dims[2] < 2 || nn > (int64_t)1 << 27) return MLQ_EINVAL;
        if (lengths && !(lengths[0] > 0.0 && lengths[1] > 0.0 && lengths[2] > 0.0)) return MLQ_EINVAL;
    } else if (dims[0] < 2 || dims[0] > 8193) {
        return MLQ_EINVAL;
    }
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->generation++;
    Level &L = ctx->levels[level];
    release_level(L);
    if (dim == 3) {
        L.dim = 3;
        if (lengths) {
            L.Lx = lengths[0];
            L.Ly = lengths[1];
            L.Lz = lengths[2];
        }
        L.g3 = mlq::make_grid3(dims[0], dims[1], dims[2], L.Lx / (dims[0] - 1), L.Ly / (dims[1] - 1),
                               L.Lz / (dims[2] - 1));
        const mlq::Grid3 &g = L.g3;
        L.n = dims[0] * dims[1] * dims[2];   // nodes; the device arrays hold g.n padded entries
        L.ne = 6 * (g.mx - 1) * (g.my - 1) * (g.mz - 1);
        L.dt = dt;
        L.nsteps = nsteps;
        MLQ_CUDA(ctx, cudaMalloc(&L.d_M3, sizeof(double) * 8 * (size_t)g.n));
        MLQ_CUDA(ctx, cudaMalloc(&L.d_lump, sizeof(double) * (size_t)g.n));
        MLQ_CUDA(ctx, mlq::launch_level3d_setup(g, L.d_M3, L.d_lump, ctx->stream));
        MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->launches++;
        L.defined = true;
        return MLQ_OK;
    }
    const int m = dims[0];
    L.dim = 2;
    L.m = m;
    L.n = m * m;
    L.ne = 2 * (m - 1) * (m - 1);
    L.h = 1.0 / (double)(m - 1);
    L.dt = dt;
    L.nsteps = nsteps;
    if (!fastdiv_make((uint32_t)m, (uint32_t)L.n, &L.divm)) return MLQ_EINVAL;
    L.defined = true;
    return MLQ_OK;
}

int mlq_add_level_mesh(mlq_ctx *ctx, int level, int64_t n, const double *xyz, int64_t ne, const int32_t *conn,
                       const double *frames, double dt, int32_t nsteps)
{
    MLQ_GUARD(ctx);
    if (!ctx || !xyz || !conn || level < 0 || level >= kMaxLevels) return MLQ_EINVAL;
    if (!(dt > 0.0) || nsteps < 0 || n < 4 || ne < 1 || n > ((int64_t)1 << 27)) return MLQ_EINVAL;
    if (ctx->scheme.ionic == 1) return MLQ_EUNSUPPORTED;   // the paper's scheme runs on 2D levels only
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    mlq_mesh *mesh = nullptr;
    const int st = mlq_mesh_create(&mesh, ctx->device, n, xyz, ne, conn, frames);
    if (st != MLQ_OK) return st;
    ctx->generation++;
    Level &L = ctx->levels[level];
    release_level(L);
    L.dim = 3;
    L.mesh = mesh;
    L.n = (int)n;
    L.ne = (int)ne;
    L.dt = dt;
    L.nsteps = nsteps;
    L.xyz_h.assign(xyz, xyz + (size_t)n * 3);
    L.conn_h.assign(conn, conn + (size_t)ne * 4);
    const int su = upload_mesh_disk(L);
    if (su != MLQ_OK) {
        release_level(L);
        return su;
    }
    L.defined = true;
    return MLQ_OK;
}

int mlq_set_initial_state(mlq_ctx *ctx, int level, const double *v0, const double *w0)
{
    MLQ_GUARD(ctx);
    if (!ctx || !v0 || level < 0 || level >= kMaxLevels || !ctx->levels[level].defined) return MLQ_EINVAL;
    ctx->generation++;
    Level &L = ctx->levels[level];
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    if (!L.d_v0) MLQ_CUDA(ctx, cudaMalloc(&L.d_v0, sizeof(double) * L.n));
    MLQ_CUDA(ctx, cudaMemcpy(L.d_v0, v0, sizeof(double) * L.n, cudaMemcpyDefault));
    if (w0) {
        if (!L.d_w0) MLQ_CUDA(ctx, cudaMalloc(&L.d_w0, sizeof(double) * L.n));
        MLQ_CUDA(ctx, cudaMemcpy(L.d_w0, w0, sizeof(double) * L.n, cudaMemcpyDefault));
    } else if (L.d_w0) {
        cudaFree(L.d_w0);
        L.d_w0 = nullptr;
    }
    return MLQ_OK;
}

int mlq_set_initial_disk(mlq_ctx *ctx, int level, double radius)
{
    MLQ_GUARD(ctx);
    if (!ctx || level < 0 || level >= kMaxLevels || !ctx->levels[level].defined || !(radius >= 0.0))
        return MLQ_EINVAL;
    ctx->generation++;
    Level &L = ctx->levels[level];
    cudaFree(L.d_v0);
    cudaFree(L.d_w0);
    L.d_v0 = L.d_w0 = nullptr;
    L.radius = radius;
    if (L.mesh) {
        MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
        return upload_mesh_disk(L);
    }
    return MLQ_OK;
}

int mlq_set_kl(mlq_ctx *ctx, int level, int K, const double *phi, const double *theta_mean)
{
    MLQ_GUARD(ctx);
    if (!ctx || !phi || K < 1 || K > kMaxK || level < 0 || level >= kMaxLevels || !ctx->levels[level].defined)
        return MLQ_EINVAL;
    ctx->generation++;
    Level &L = ctx->levels[level];
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    if (L.mesh) {
        // the general mesh's table (host copies: phi and theta_mean may be device pointers)
        std::vector<double> ph((size_t)L.ne * K), tm(theta_mean ? (size_t)L.ne : 0);
        MLQ_CUDA(ctx, cudaMemcpy(ph.data(), phi, sizeof(double) * ph.size(), cudaMemcpyDefault));
        if (theta_mean) MLQ_CUDA(ctx, cudaMemcpy(tm.data(), theta_mean, sizeof(double) * tm.size(), cudaMemcpyDefault));
        const int st = mlq_mesh_set_kl(L.mesh, K, ph.data(), theta_mean ? tm.data() : nullptr);
        if (st != MLQ_OK) return st;
        L.K = K;
        return MLQ_OK;
    }
    cudaFree(L.d_phi);
    cudaFree(L.d_theta_mean);
    L.d_phi = L.d_theta_mean = nullptr;
    MLQ_CUDA(ctx, cudaMalloc(&L.d_phi, sizeof(double) * (size_t)L.ne * K));
    MLQ_CUDA(ctx, cudaMemcpy(L.d_phi, phi, sizeof(double) * (size_t)L.ne * K, cudaMemcpyDefault));
    // TF32 split of the table for the tensor-core synthesis: hi = the value
    // rounded to FP32 with the low 13 mantissa bits cleared, lo = remainder
    {
        cudaFree(L.d_phi_hi);
        cudaFree(L.d_phi_lo);
        L.d_phi_hi = L.d_phi_lo = nullptr;
        L.Kp = (K + 7) / 8 * 8;
        std::vector<double> hp((size_t)L.ne * K);
        MLQ_CUDA(ctx, cudaMemcpy(hp.data(), L.d_phi, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost));
        std::vector<float> hi((size_t)L.ne * L.Kp, 0.0f), lo((size_t)L.ne * L.Kp, 0.0f);
        for (int64_t e = 0; e < L.ne; ++e)
            for (int k = 0; k < K; ++k) {
                const float x = (float)hp[(size_t)e * K + k];
                uint32_t b;
                std::memcpy(&b, &x, 4);
                b &= 0xFFFFE000u;
                float h;
                std::memcpy(&h, &b, 4);
                hi[(size_t)e * L.Kp + k] = h;
                lo[(size_t)e * L.Kp + k] = x - h;
            }
        MLQ_CUDA(ctx, cudaMalloc(&L.d_phi_hi, sizeof(float) * hi.size()));
        MLQ_CUDA(ctx, cudaMalloc(&L.d_phi_lo, sizeof(float) * lo.size()));
        MLQ_CUDA(ctx, cudaMemcpy(L.d_phi_hi, hi.data(), sizeof(float) * hi.size(), cudaMemcpyHostToDevice));
        MLQ_CUDA(ctx, cudaMemcpy(L.d_phi_lo, lo.data(), sizeof(float) * lo.size(), cudaMemcpyHostToDevice));
    }
    if (theta_mean) {
        MLQ_CUDA(ctx, cudaMalloc(&L.d_theta_mean, sizeof(double) * (size_t)L.ne));
        MLQ_CUDA(ctx, cudaMemcpy(L.d_theta_mean, theta_mean, sizeof(double) * (size_t)L.ne, cudaMemcpyDefault));
    }
    L.K = K;
    return MLQ_OK;
}

int mlq_synthesize(mlq_ctx *ctx, int level, int64_t S, const double *xi, double *cs2_out)
{
    MLQ_GUARD(ctx);
    if (!ctx || !xi || !cs2_out || S < 1 || S > 65535) return MLQ_EINVAL;
    if (check_level(ctx, level) != MLQ_OK) return MLQ_EINVAL;
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    const Level &L = ctx->levels[level];
    if (L.mesh) return synthesize_mesh(ctx, level, S, xi, cs2_out);
    const size_t out_b = align_up((size_t)S * L.ne * 16, 256), xi_b = align_up((size_t)S * L.K * 8, 256);
    int st = ensure_workspace(ctx, out_b + xi_b);
    if (st != MLQ_OK) return st;
    double *cs2 = (double *)ctx->ws;
    const double *d_xi = xi;
    if (!is_device_ptr(xi)) {
        double *dx = (double *)((char *)ctx->ws + out_b);
        MLQ_CUDA(ctx, cudaMemcpyAsync(dx, xi, sizeof(double) * S * L.K, cudaMemcpyHostToDevice, ctx->stream));
        d_xi = dx;
    }
    if ((st = launch_synthesis(ctx, L, d_xi, (int)S, cs2, ctx->stream)) != MLQ_OK) return st;
    MLQ_CUDA(ctx, cudaMemcpyAsync(cs2_out, cs2, (size_t)S * L.ne * 16, cudaMemcpyDefault, ctx->stream));
    MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}

int mlq_workspace_bytes(mlq_ctx *ctx, int level, int64_t S, int with_coarse, size_t *bytes)
{
    MLQ_GUARD(ctx);
    if (!ctx || !bytes || S < 0) return MLQ_EINVAL;
    if (check_level(ctx, level) != MLQ_OK) return MLQ_EINVAL;
    size_t t = member_bytes(ctx, ctx->levels[level], S);
    if (with_coarse) {
        if (check_level(ctx, level - 1) != MLQ_OK) return MLQ_EINVAL;
        t += member_bytes(ctx, ctx->levels[level - 1], S);
    }
    t += align_up((size_t)S * ctx->levels[level].K * 8, 256);  // xi staging
    t += align_up((size_t)S * 8, 256) + align_up((size_t)S * 4, 256) + 256;  // y, status, sums
    *bytes = t;
    return MLQ_OK;
}

int mlq_solve(mlq_ctx *ctx, int level, int64_t S, const double *xi, int with_coarse, double *q_fine,
              double *q_coarse, double *y, int32_t *status, int32_t *iters)
{
    MLQ_GUARD(ctx);
    if (!ctx || !xi || S < 0 || S > 65535) return MLQ_EINVAL;
    if (check_level(ctx, level) != MLQ_OK) return MLQ_EINVAL;
    if (with_coarse) {
        if (check_level(ctx, level - 1) != MLQ_OK) return MLQ_EINVAL;
        if (ctx->levels[level - 1].K != ctx->levels[level].K) return MLQ_EINVAL;
    }
    if (S == 0) return MLQ_OK;
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->nmembers = 0;
    const int K = ctx->levels[level].K;
    size_t need = 0;
    mlq_workspace_bytes(ctx, level, S, with_coarse, &need);
    int st = ensure_workspace(ctx, need);
    if (st != MLQ_OK) return st;
    char *cur = (char *)ctx->ws;
    Member mf, mc;
    mf.level = level;
    mf.S = S;
    member_carve(ctx, ctx->levels[level], mf, cur);
    if (with_coarse) {
        mc.level = level - 1;
        mc.S = S;
        member_carve(ctx, ctx->levels[level - 1], mc, cur);
    }
    double *ybuf = (double *)cur;
    cur += align_up((size_t)S * 8, 256);
    double *sums = (double *)cur;
    cur += 256;
    int32_t *stbuf = (int32_t *)cur;
    cur += align_up((size_t)S * 4, 256);
    // xi on the device
    const double *d_xi = xi;
    if ((st = carve_check(ctx, cur, is_device_ptr(xi) ? 0 : (size_t)S * K * 8)) != MLQ_OK) return st;
    if (!is_device_ptr(xi)) {
        double *dx = (double *)cur;
        MLQ_CUDA(ctx, cudaMemcpyAsync(dx, xi, sizeof(double) * S * K, cudaMemcpyHostToDevice, ctx->stream));
        d_xi = dx;
    }
    mf.d_xi = d_xi;
    mc.d_xi = d_xi;
    // fork: fine on pool[0], coarse on pool[1]
    if (ctx->profile) MLQ_CUDA(ctx, cudaEventRecord(ctx->ev_start, ctx->stream));
    MLQ_CUDA(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
    const int nm = with_coarse ? 2 : 1;
    for (int k = 0; k < nm; ++k) {
        MLQ_CUDA(ctx, cudaStreamWaitEvent(ctx->pool[k], ctx->ev_fork, 0));
        st = launch_member(ctx, k == 0 ? mf : mc, ctx->pool[k], k, k);
        if (st != MLQ_OK) return st;
        MLQ_CUDA(ctx, cudaEventRecord(ctx->ev_join[k], ctx->pool[k]));
        MLQ_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join[k], 0));
    }
    // K7
    mlq::level_sums_kernel<<<1, 1024, 0, ctx->stream>>>(mf.q, with_coarse ? mc.q : nullptr, S, ybuf, sums);
    MLQ_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    mlq::merge_status_kernel<<<(unsigned)((S + 255) / 256), 256, 0, ctx->stream>>>(
        mf.status, with_coarse ? mc.status : nullptr, S, stbuf);
    MLQ_CUDA(ctx, cudaGetLastError());
    ctx->launches++;
    if ((st = copy_out(ctx, q_fine, mf.q, S * 8, ctx->stream)) != MLQ_OK) return st;
    if (with_coarse && (st = copy_out(ctx, q_coarse, mc.q, S * 8, ctx->stream)) != MLQ_OK) return st;
    if ((st = copy_out(ctx, y, ybuf, S * 8, ctx->stream)) != MLQ_OK) return st;
    if ((st = copy_out(ctx, status, stbuf, S * 4, ctx->stream)) != MLQ_OK) return st;
    if ((st = copy_out(ctx, iters, mf.iters, S * 4, ctx->stream)) != MLQ_OK) return st;
    MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}

int mlq_solve_state(mlq_ctx *ctx, int level, int64_t S, const double *xi, double *v_out, double *w_out,
                    double *q_out, int32_t *status)
{
    MLQ_GUARD(ctx);
    if (!ctx || !xi || S < 0 || S > 65535) return MLQ_EINVAL;
    if (check_level(ctx, level) != MLQ_OK) return MLQ_EINVAL;
    if (S == 0) return MLQ_OK;
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->nmembers = 0;
    const Level &L = ctx->levels[level];
    const int K = L.K;
    size_t need = 0;
    mlq_workspace_bytes(ctx, level, S, 0, &need);
    int st = ensure_workspace(ctx, need);
    if (st != MLQ_OK) return st;
    char *cur = (char *)ctx->ws;
    Member mf;
    mf.level = level;
    mf.S = S;
    member_carve(ctx, L, mf, cur);
    cur += align_up((size_t)S * 8, 256) + 256 + align_up((size_t)S * 4, 256);  // as mlq_solve's carve
    const double *d_xi = xi;
    if ((st = carve_check(ctx, cur, is_device_ptr(xi) ? 0 : (size_t)S * K * 8)) != MLQ_OK) return st;
    if (!is_device_ptr(xi)) {
        double *dx = (double *)cur;
        MLQ_CUDA(ctx, cudaMemcpyAsync(dx, xi, sizeof(double) * S * K, cudaMemcpyHostToDevice, ctx->stream));
        d_xi = dx;
    }
    mf.d_xi = d_xi;
    MLQ_CUDA(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
    MLQ_CUDA(ctx, cudaStreamWaitEvent(ctx->pool[0], ctx->ev_fork, 0));
    if ((st = launch_member(ctx, mf, ctx->pool[0], 0, 0)) != MLQ_OK) return st;
    MLQ_CUDA(ctx, cudaEventRecord(ctx->ev_join[0], ctx->pool[0]));
    MLQ_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join[0], 0));
    // where the kernels leave the state after the last block: the ring kernels
    // (multigrid and 3D) keep v_j in buffer j mod kVRing, the others update v
    // in place; w alternates between two buffers, one per block.  The
    // general-mesh solver updates both in place ([S][n] FP64).
    const size_t SN = (size_t)S * (L.mesh ? (size_t)L.n : stored(L));
    const bool ring = !L.mesh && (L.dim == 3 || choose_launch(ctx, L, S).mg);
    const double *vfin = L.mesh ? mf.mws.v : mf.v + (ring ? (size_t)(L.nsteps % mlq::kVRing) * SN : 0);
    const double *wfin = L.mesh ? mf.mws.w : mf.w + (size_t)(L.nsteps & 1) * SN;
    if (L.dim == 3 && !L.mesh) {
        // the real entries of every padded row, S x my x mz rows of mx
        const mlq::Grid3 &g = L.g3;
        const size_t rows = (size_t)S * g.my * g.mz;
        for (int t = 0; t < 2; ++t) {
            double *dst = t == 0 ? v_out : w_out;
            const double *src = t == 0 ? vfin : wfin;
            if (!dst) continue;
            MLQ_CUDA(ctx, cudaMemcpy2DAsync(dst, sizeof(double) * g.mx, src, sizeof(double) * g.px,
                                            sizeof(double) * g.mx, rows, cudaMemcpyDefault, ctx->stream));
        }
    } else {
        if ((st = copy_out(ctx, v_out, vfin, SN * 8, ctx->stream)) != MLQ_OK) return st;
        if ((st = copy_out(ctx, w_out, wfin, SN * 8, ctx->stream)) != MLQ_OK) return st;
    }
    if ((st = copy_out(ctx, q_out, mf.q, S * 8, ctx->stream)) != MLQ_OK) return st;
    if ((st = copy_out(ctx, status, mf.status, S * 4, ctx->stream)) != MLQ_OK) return st;
    MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}

}  // extern "C"

namespace {

// The simplex of a structured level holding point x and the point's
// barycentric weights there (nodes [4], weights [4]; 2D: the 4th entry
// repeats node 0 with weight 0).  The cell is the one whose lower corner is
// floor(x / h) (clamped to the mesh), the simplex the first of the cell, in
// the mesh convention's order, that contains the point.  false if x lies
// outside the domain by more than 1e-12 of its extent.
bool locate_point(const Level &L, const double *x, int *node, double *w)
{
    if (L.dim == 2) {
        const int m = L.m;
        const double f[2] = {x[0] / L.h, x[1] / L.h};
        int c[2];
        double t[2];
        for (int a = 0; a < 2; ++a) {
            if (!(x[a] >= -1e-12 && x[a] <= 1.0 + 1e-12)) return false;
            c[a] = std::min(std::max((int)std::floor(f[a]), 0), m - 2);
            t[a] = std::min(std::max(f[a] - c[a], 0.0), 1.0);
        }
        const int n00 = c[0] + m * c[1];
        if (t[1] <= t[0]) {   // element 2c: (i,j) (i+1,j) (i+1,j+1)
            node[0] = n00; node[1] = n00 + 1; node[2] = n00 + m + 1;
            w[0] = 1.0 - t[0]; w[1] = t[0] - t[1]; w[2] = t[1];
        } else {              // element 2c+1: (i,j) (i+1,j+1) (i,j+1)
            node[0] = n00; node[1] = n00 + m + 1; node[2] = n00 + m;
            w[0] = 1.0 - t[1]; w[1] = t[0]; w[2] = t[1] - t[0];
        }
        node[3] = n00;
        w[3] = 0.0;
        return true;
    }
    const mlq::Grid3 &g = L.g3;
    const int mm[3] = {g.mx, g.my, g.mz};
    const double len[3] = {L.Lx, L.Ly, L.Lz}, hh[3] = {g.hx, g.hy, g.hz};
    int c[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        if (!(x[a] >= -1e-12 * len[a] && x[a] <= len[a] * (1.0 + 1e-12))) return false;
        const double f = x[a] / hh[a];
        c[a] = std::min(std::max((int)std::floor(f), 0), mm[a] - 2);
        t[a] = std::min(std::max(f - c[a], 0.0), 1.0);
    }
    // tetrahedron s of the cell holds the points whose local coordinates fall
    // along its step axes: t[a0] >= t[a1] >= t[a2]
    int s = 0;
    for (; s < 6; ++s) {
        const int a0 = mlq::kuhn_axis(s, 0), a1 = mlq::kuhn_axis(s, 1), a2 = mlq::kuhn_axis(s, 2);
        if (t[a0] >= t[a1] && t[a1] >= t[a2]) break;
    }
    const int a0 = mlq::kuhn_axis(s, 0), a1 = mlq::kuhn_axis(s, 1), a2 = mlq::kuhn_axis(s, 2);
    const double lam[4] = {1.0 - t[a0], t[a0] - t[a1], t[a1] - t[a2], t[a2]};
    for (int q = 0; q < 4; ++q) {
        const int msk = mlq::kuhn_vertex(s, q);
        node[q] = (int)mlq::grid3_index(g, c[0] + (msk & 1), c[1] + ((msk >> 1) & 1), c[2] + ((msk >> 2) & 1));
        w[q] = lam[q];
    }
    return true;
}

}  // namespace

extern "C" {

int mlq_set_points(mlq_ctx *ctx, int level, int np, const double *pts, double u_th)
{
    MLQ_GUARD(ctx);
    if (!ctx || level < 0 || level >= kMaxLevels || !ctx->levels[level].defined) return MLQ_EINVAL;
    if (np < 0 || np > mlq::kMaxPoints || (np > 0 && !pts) || !std::isfinite(u_th)) return MLQ_EINVAL;
    Level &L = ctx->levels[level];
    std::vector<int> nd(4 * (size_t)std::max(np, 1));
    std::vector<double> wt(4 * (size_t)std::max(np, 1));
    if (L.mesh) {
        // general mesh: the first tetrahedron holding each point; a point
        // whose best tetrahedron still has a barycentric coordinate below
        // -1e-9 lies outside the mesh
        std::vector<int64_t> el((size_t)std::max(np, 1));
        const int sl = mlq::locate_points(3, (int64_t)L.n, L.xyz_h.data(), (int64_t)L.ne, L.conn_h.data(), np, pts,
                                          el.data(), wt.data());
        if (sl != MLQ_OK) return sl;
        for (int p = 0; p < np; ++p)
            for (int a = 0; a < 4; ++a) {
                if (!(wt[4 * p + a] >= -1e-9)) return MLQ_EINVAL;
                nd[4 * p + a] = L.conn_h[(size_t)el[(size_t)p] * 4 + a];
            }
    } else {
        for (int p = 0; p < np; ++p)
            if (!locate_point(L, pts + (size_t)p * L.dim, &nd[4 * p], &wt[4 * p])) return MLQ_EINVAL;
    }
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(L.d_pt_node);
    cudaFree(L.d_pt_w);
    L.d_pt_node = nullptr;
    L.d_pt_w = nullptr;
    L.npts = 0;
    if (np == 0) return MLQ_OK;
    MLQ_CUDA(ctx, cudaMalloc(&L.d_pt_node, sizeof(int) * 4 * (size_t)np));
    MLQ_CUDA(ctx, cudaMalloc(&L.d_pt_w, sizeof(double) * 4 * (size_t)np));
    MLQ_CUDA(ctx, cudaMemcpy(L.d_pt_node, nd.data(), sizeof(int) * 4 * (size_t)np, cudaMemcpyHostToDevice));
    MLQ_CUDA(ctx, cudaMemcpy(L.d_pt_w, wt.data(), sizeof(double) * 4 * (size_t)np, cudaMemcpyHostToDevice));
    L.npts = np;
    L.u_th = u_th;
    return MLQ_OK;
}

int mlq_solve_points(mlq_ctx *ctx, int level, int64_t S, const double *xi, double *trace, double *act,
                     double *q_out, int32_t *status)
{
    MLQ_GUARD(ctx);
    if (!ctx || !xi || S < 0 || S > 65535) return MLQ_EINVAL;
    if (check_level(ctx, level) != MLQ_OK || ctx->levels[level].npts < 1) return MLQ_EINVAL;
    if (S == 0) return MLQ_OK;
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->nmembers = 0;
    const Level &L = ctx->levels[level];
    const int K = L.K, np = L.npts;
    const size_t tr_bytes = align_up((size_t)S * np * (L.nsteps + 1) * 8, 256);
    const size_t ac_bytes = align_up((size_t)S * np * 8, 256);
    size_t need = 0;
    mlq_workspace_bytes(ctx, level, S, 0, &need);
    int st = ensure_workspace(ctx, need + tr_bytes + ac_bytes);
    if (st != MLQ_OK) return st;
    char *cur = (char *)ctx->ws;
    Member mf;
    mf.level = level;
    mf.S = S;
    member_carve(ctx, L, mf, cur);
    cur += align_up((size_t)S * 8, 256) + 256 + align_up((size_t)S * 4, 256);  // as mlq_solve's carve
    const double *d_xi = xi;
    const size_t xi_bytes = is_device_ptr(xi) ? 0 : align_up((size_t)S * K * 8, 256);
    if ((st = carve_check(ctx, cur, xi_bytes + tr_bytes + ac_bytes)) != MLQ_OK) return st;
    if (xi_bytes) {
        double *dx = (double *)cur;
        cur += xi_bytes;
        MLQ_CUDA(ctx, cudaMemcpyAsync(dx, xi, sizeof(double) * S * K, cudaMemcpyHostToDevice, ctx->stream));
        d_xi = dx;
    }
    double *d_tr = (double *)cur;
    cur += tr_bytes;
    double *d_act = (double *)cur;
    mf.d_xi = d_xi;
    mf.pq.npts = np;
    mf.pq.node = L.d_pt_node;
    mf.pq.w = L.d_pt_w;
    mf.pq.u_th = L.u_th;
    mf.pq.trace = d_tr;
    mf.pq.act = d_act;
    MLQ_CUDA(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
    MLQ_CUDA(ctx, cudaStreamWaitEvent(ctx->pool[0], ctx->ev_fork, 0));
    if ((st = launch_member(ctx, mf, ctx->pool[0], 0, 0)) != MLQ_OK) return st;
    MLQ_CUDA(ctx, cudaEventRecord(ctx->ev_join[0], ctx->pool[0]));
    MLQ_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join[0], 0));
    if ((st = copy_out(ctx, trace, d_tr, (size_t)S * np * (L.nsteps + 1) * 8, ctx->stream)) != MLQ_OK) return st;
    if ((st = copy_out(ctx, act, d_act, (size_t)S * np * 8, ctx->stream)) != MLQ_OK) return st;
    if ((st = copy_out(ctx, q_out, mf.q, S * 8, ctx->stream)) != MLQ_OK) return st;
    if ((st = copy_out(ctx, status, mf.status, S * 4, ctx->stream)) != MLQ_OK) return st;
    MLQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}

int mlq_estimate(mlq_ctx *ctx, int L, const int64_t *N, const double *const *xi, double *mean_out,
                 double *var_out, double *rmse_out, double *const *y_out)
{
    MLQ_GUARD(ctx);
    if (!ctx || !N || !xi || !mean_out || L < 0 || L >= kMaxLevels) return MLQ_EINVAL;
    if (2 * (L + 1) > kStreams) return MLQ_EUNSUPPORTED;
    for (int l = 0; l <= L; ++l) {
        if (check_level(ctx, l) != MLQ_OK || N[l] < 2 || N[l] > 65535 || !xi[l]) return MLQ_EINVAL;
        if (ctx->levels[l].K != ctx->levels[0].K) return MLQ_EINVAL;
    }
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->nmembers = 0;
    const int K = ctx->levels[0].K;
    // With more members than lanes, the two members on the coarsest mesh
    // (the fine member of pair 0 and the coarse member of pair 1) run as one
    // launch of N_0 + N_1 samples, when the launch shape is the same for
    // each alone and for both (every sample is then solved exactly as in
    // its own member): no member waits for another's lane.
    const bool merge0 = L >= 1 && 2 * L + 1 > kLanes && N[0] + N[1] <= 65535 &&
                        same_shape(choose_launch(ctx, ctx->levels[0], N[0]), choose_launch(ctx, ctx->levels[0], N[1])) &&
                        same_shape(choose_launch(ctx, ctx->levels[0], N[0]),
                                   choose_launch(ctx, ctx->levels[0], N[0] + N[1]));
    size_t need = 4096;
    for (int l = 0; l <= L; ++l) {
        need += member_bytes(ctx, ctx->levels[l], N[l]);
        if (l > 0) need += member_bytes(ctx, ctx->levels[l - 1], N[l]);
        need += align_up((size_t)N[l] * 8, 256) * 2 + align_up((size_t)N[l] * K * 8, 256);
    }
    if (merge0) need += member_bytes(ctx, ctx->levels[0], N[0] + N[1]) + align_up((size_t)(N[0] + N[1]) * K * 8, 256);
    int st = ensure_workspace(ctx, need);
    if (st != MLQ_OK) return st;
    char *cur = (char *)ctx->ws;
    std::vector<Member> fine(L + 1), coarse(L + 1);
    std::vector<double *> ybuf(L + 1);
    double *sums = (double *)cur;
    cur += align_up(sizeof(double) * 2 * (L + 1), 256);
    for (int l = 0; l <= L; ++l) {
        fine[l].level = l;
        fine[l].S = N[l];
        member_carve(ctx, ctx->levels[l], fine[l], cur);
        if (l > 0) {
            coarse[l].level = l - 1;
            coarse[l].S = N[l];
            member_carve(ctx, ctx->levels[l - 1], coarse[l], cur);
        }
        ybuf[l] = (double *)cur;
        cur += align_up((size_t)N[l] * 8, 256);
        const double *d_xi = xi[l];
        if ((st = carve_check(ctx, cur, is_device_ptr(xi[l]) ? 0 : (size_t)N[l] * K * 8)) != MLQ_OK) return st;
        if (!is_device_ptr(xi[l])) {
            double *dx = (double *)cur;
            cur += align_up((size_t)N[l] * K * 8, 256);
            MLQ_CUDA(ctx, cudaMemcpyAsync(dx, xi[l], sizeof(double) * N[l] * K, cudaMemcpyHostToDevice,
                                          ctx->stream));
            d_xi = dx;
        }
        fine[l].d_xi = coarse[l].d_xi = d_xi;
    }
    Member m0;   // the merged coarsest-mesh member: samples of pair 0, then of pair 1
    double *xi01 = nullptr;
    if (merge0) {
        m0.level = 0;
        m0.S = N[0] + N[1];
        member_carve(ctx, ctx->levels[0], m0, cur);
        if ((st = carve_check(ctx, cur, (size_t)m0.S * K * 8)) != MLQ_OK) return st;
        xi01 = (double *)cur;
        cur += align_up((size_t)m0.S * K * 8, 256);
        m0.d_xi = xi01;
        fine[0].q = m0.q;
        fine[0].iters = m0.iters;
        fine[0].status = m0.status;
        coarse[1].q = m0.q + N[0];
        coarse[1].iters = m0.iters + N[0];
        coarse[1].status = m0.status + N[0];
    }
    // launch order: largest levels first (slot = lane index)
    std::vector<std::pair<const Member *, int>> order;
    for (int l = L; l >= 0; --l)
        for (int k = 0; k < (l > 0 ? 2 : 1); ++k) {
            if (merge0 && l == 0) continue;
            if (merge0 && l == 1 && k == 1) order.push_back({&m0, 1});
            else order.push_back({k == 0 ? &fine[l] : &coarse[l], k});
        }
    // CUDA graph: capture the whole estimate once, replay while unchanged
    bool use_graph = ctx->opt.graphs != 0 && ctx->stream != nullptr;
    for (int l = 0; l <= L && use_graph; ++l) {
        if (!is_device_ptr(xi[l])) use_graph = false;
        if (y_out && y_out[l] && !is_device_ptr(y_out[l])) use_graph = false;
    }
    std::vector<uint64_t> key;
    if (use_graph) {
        key.push_back(ctx->generation);
        key.push_back((uint64_t)L);
        key.push_back((uint64_t)(uintptr_t)ctx->ws);
        key.push_back((uint64_t)ctx->profile);
        for (int l = 0; l <= L; ++l) {
            key.push_back((uint64_t)N[l]);
            key.push_back((uint64_t)(uintptr_t)xi[l]);
            key.push_back((uint64_t)(uintptr_t)(y_out ? y_out[l] : nullptr));
        }
        if (ctx->graph_exec && key == ctx->graph_key) {
            ctx->nmembers = 0;
            for (size_t sid = 0; sid < order.size(); ++sid)
                if (ctx->profile) launch_member_profile_only(ctx, *order[sid].first, (int)sid, order[sid].second);
            MLQ_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->stream));
            ctx->launches += ctx->graph_launches;
            return finish_estimate(ctx, L, N, mean_out, var_out, rmse_out);
        }
        if (ctx->graph_exec) {
            cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
        }
        MLQ_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
    }
    const int64_t launches_before = ctx->launches;
    auto abort_capture = [&](int code) {
        if (ctx->capturing) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(ctx->stream, &g);
            if (g) cudaGraphDestroy(g);
            ctx->capturing = false;
            cudaGetLastError();
        }
        return code;
    };
    if (ctx->profile && cudaEventRecordWithFlags(ctx->ev_start, ctx->stream,
                                                 ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault) !=
                            cudaSuccess)
        return abort_capture(MLQ_ECUDA);
    if (merge0) {   // the merged member's samples, contiguous (inside the capture: replays recopy)
        if (cudaMemcpyAsync(xi01, fine[0].d_xi, sizeof(double) * N[0] * K, cudaMemcpyDeviceToDevice, ctx->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(xi01 + (size_t)N[0] * K, coarse[1].d_xi, sizeof(double) * N[1] * K,
                            cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
            return abort_capture(MLQ_ECUDA);
    }
    if (cudaEventRecord(ctx->ev_fork, ctx->stream) != cudaSuccess) return abort_capture(MLQ_ECUDA);
    // every member's set-up first (short kernels), joined, then the solves,
    // largest levels first on the higher-priority streams: the finest level
    // is the critical path and takes freed SMs first
    for (int phase : {kSetup, kSolve}) {
        if (phase == kSolve && cudaEventRecord(ctx->ev_fork, ctx->stream) != cudaSuccess)
            return abort_capture(MLQ_ECUDA);
        for (int sid = 0; sid < (int)order.size(); ++sid) {
            // the device has kLanes hardware queues by default: members
            // past the last lane (the smallest) run in turn on it instead
            // of sharing a queue with a large member
            cudaStream_t s = ctx->pool[std::min(sid, kLanes - 1)];
            if (cudaStreamWaitEvent(s, ctx->ev_fork, 0) != cudaSuccess) return abort_capture(MLQ_ECUDA);
            st = launch_member(ctx, *order[sid].first, s, sid, order[sid].second, phase);
            if (st != MLQ_OK) return abort_capture(st);
            if (cudaEventRecord(ctx->ev_join[sid], s) != cudaSuccess ||
                cudaStreamWaitEvent(ctx->stream, ctx->ev_join[sid], 0) != cudaSuccess)
                return abort_capture(MLQ_ECUDA);
        }
    }
    for (int l = 0; l <= L; ++l) {
        mlq::level_sums_kernel<<<1, 1024, 0, ctx->stream>>>(fine[l].q, l > 0 ? coarse[l].q : nullptr, N[l],
                                                              ybuf[l], sums + 2 * l);
        if (cudaGetLastError() != cudaSuccess) return abort_capture(MLQ_ECUDA);
        ctx->launches++;
        if (y_out && y_out[l]) {
            if ((st = copy_out(ctx, y_out[l], ybuf[l], (size_t)N[l] * 8, ctx->stream)) != MLQ_OK)
                return abort_capture(st);
        }
    }
    if (cudaMemcpyAsync(ctx->h_sums, sums, sizeof(double) * 2 * (L + 1), cudaMemcpyDeviceToHost, ctx->stream) !=
        cudaSuccess)
        return abort_capture(MLQ_ECUDA);
    if (ctx->capturing) {
        cudaGraph_t g = nullptr;
        ctx->capturing = false;
        MLQ_CUDA(ctx, cudaStreamEndCapture(ctx->stream, &g));
        // kernel nodes keep the priority of the stream they were captured from
        cudaError_t e = cudaGraphInstantiate(&ctx->graph_exec, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ctx->graph_exec = nullptr;
            ctx->cuda_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
            return MLQ_ECUDA;
        }
        ctx->graph_key = key;
        ctx->graph_launches = ctx->launches - launches_before;
        MLQ_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    }
    return finish_estimate(ctx, L, N, mean_out, var_out, rmse_out);
}

int mlq_estimate_adaptive(mlq_ctx *ctx, int L, double eps, int64_t n_pilot, const int64_t *Nmax,
                          const double *const *xi, int64_t *N_out, double *mean_out, double *var_out,
                          double *rmse_out)
try {
    MLQ_GUARD(ctx);
    if (!ctx || !Nmax || !xi || !N_out || !mean_out || L < 0 || L >= kMaxLevels || !(eps > 0.0) || n_pilot < 2)
        return MLQ_EINVAL;
    for (int l = 0; l <= L; ++l) {
        if (check_level(ctx, l) != MLQ_OK || Nmax[l] < n_pilot || !xi[l]) return MLQ_EINVAL;
        if (ctx->levels[l].K != ctx->levels[0].K) return MLQ_EINVAL;
    }
    const int K = ctx->levels[0].K;
    // cost per sample of level pair l: the DOF-steps of its members
    std::vector<double> cost(L + 1), var(L + 1);
    for (int l = 0; l <= L; ++l) {
        const Level &F = ctx->levels[l];
        cost[l] = (double)F.n * F.nsteps;
        if (l > 0) cost[l] += (double)ctx->levels[l - 1].n * ctx->levels[l - 1].nsteps;
    }
    std::vector<std::vector<double>> y(L + 1);
    std::vector<int64_t> N(L + 1, 0), want(L + 1);
    for (int l = 0; l <= L; ++l) want[l] = n_pilot;
    std::vector<double> yb, qf, qc;
    std::vector<int32_t> stb;
    // solve samples [N_l, want_l) of every level, in index order and in
    // pieces of at most 65535
    auto top_up = [&]() -> int {
        for (int l = 0; l <= L; ++l) {
            while (N[l] < want[l]) {
                const int64_t c = std::min<int64_t>(want[l] - N[l], 65535);
                yb.assign(c, 0.0);
                stb.assign(c, 0);
                const int st = mlq_solve(ctx, l, c, xi[l] + (size_t)N[l] * K, l > 0, nullptr, nullptr, yb.data(),
                                         stb.data(), nullptr);
                if (st != MLQ_OK) return st;
                y[l].insert(y[l].end(), yb.begin(), yb.end());
                N[l] += c;
            }
        }
        return MLQ_OK;
    };
    for (int round = 0; round < 16; ++round) {
        int st = top_up();
        if (st != MLQ_OK) return st;
        std::vector<const double *> yp(L + 1);
        for (int l = 0; l <= L; ++l) yp[l] = y[l].data();
        double mean = 0.0, rmse = 0.0;
        if ((st = mlq_mlmc_combine(L, N.data(), yp.data(), &mean, var.data(), &rmse)) != MLQ_OK) return st;
        // the allocation for eps from the current variance estimates, within the pools
        std::vector<double> vpos(var);
        for (double &v : vpos) v = std::max(v, 1e-300);
        std::vector<int64_t> alloc(L + 1);
        if ((st = mlq_mlmc_allocation(L, vpos.data(), cost.data(), eps, n_pilot, alloc.data())) != MLQ_OK) return st;
        bool grow = false;
        for (int l = 0; l <= L; ++l) {
            want[l] = std::min(std::max(alloc[l], N[l]), Nmax[l]);
            grow = grow || want[l] > N[l];
        }
        if (!grow) {
            for (int l = 0; l <= L; ++l) {
                N_out[l] = N[l];
                if (var_out) var_out[l] = var[l];
            }
            *mean_out = mean;
            if (rmse_out) *rmse_out = rmse;
            return MLQ_OK;
        }
    }
    return MLQ_ETIMEOUT;   // the allocation kept growing: more rounds than the loop allows
} catch (const std::bad_alloc &) {
    return MLQ_ENOMEM;
}

int mlq_set_profiling(mlq_ctx *ctx, int enable)
{
    MLQ_GUARD(ctx);
    if (!ctx) return MLQ_EINVAL;
    ctx->profile = enable != 0;
    return MLQ_OK;
}

int mlq_member_profile(mlq_ctx *ctx, int max_members, int *count, mlq_member_stats *out)
{
    MLQ_GUARD(ctx);
    if (!ctx || !count || (max_members > 0 && !out)) return MLQ_EINVAL;
    if (!ctx->profile) return MLQ_EINVAL;
    MLQ_CUDA(ctx, cudaSetDevice(ctx->device));
    const int nm = std::min(ctx->nmembers, max_members);
    *count = ctx->nmembers;
    std::vector<int32_t> it;
    for (int k = 0; k < nm; ++k) {
        mlq_member_stats &o = out[k];
        float ms = 0.0f;
        MLQ_CUDA(ctx, cudaEventSynchronize(ctx->ev_t1[k]));
        MLQ_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_t0[k], ctx->ev_t1[k]));
        o.kernel_ms = ms;
        MLQ_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_start, ctx->ev_t0[k]));
        o.start_ms = ms;
        MLQ_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_start, ctx->ev_t1[k]));
        o.end_ms = ms;
        o.level = ctx->prof_level[k];
        o.coarse = ctx->prof_coarse[k];
        o.cluster = ctx->prof_cs[k];
        o.resident = ctx->prof_resident[k];
        o.threads = ctx->prof_threads[k];
        o.npt = ctx->prof_npt[k];
        o.samples = ctx->prof_samples[k];
        o.nodes = ctx->prof_nodes[k];
        o.steps = ctx->prof_steps[k];
        it.resize((size_t)o.samples);
        MLQ_CUDA(ctx, cudaMemcpy(it.data(), ctx->prof_iters_dev[k], sizeof(int32_t) * o.samples,
                                 cudaMemcpyDeviceToHost));
        int64_t tot = 0;
        for (int32_t x : it) tot += x;
        o.cg_iterations = tot;
    }
    return MLQ_OK;
}

int mlq_autotune(mlq_ctx *ctx, int level, int64_t S, const double *xi, int probe_steps, int *cluster_out,
                 int *threads_out, double *ms_out)
{
    MLQ_GUARD(ctx);
    if (!ctx || !xi || S < 1 || probe_steps < 1) return MLQ_EINVAL;
    if (check_level(ctx, level) != MLQ_OK) return MLQ_EINVAL;
    if (ctx->opt.precision != MLQ_MIXED || ctx->opt.storage == 2) return MLQ_EUNSUPPORTED;
    Level &L = ctx->levels[level];
    if (L.dim == 3) return MLQ_EUNSUPPORTED;
    std::vector<Shape> cand = ctx->opt.precond == 1 ? mg_candidates(ctx, L) : reg_candidates(ctx, L);
    if (cand.empty()) return MLQ_EUNSUPPORTED;
    // also try the next nodes-per-thread variant of each cluster size
    const size_t nbase = cand.size();
    for (size_t k = 0; k < nbase; ++k) {
        const Shape c = cand[k];
        for (int npt : kNpt) {
            if (npt <= c.npt) continue;
            const int nmax = c.mg ? mlq::mg_plan(L.m, c.cs).lv[0].rows_max * L.m : mlq::reg_plan(L.m, c.cs).nmax;
            int th = ((nmax + npt - 1) / npt + 31) / 32 * 32;
            if (th < 32) th = 32;
            if (th > npt_max_threads(npt)) continue;
            if (c.mg && npt > 12) break;
            Shape sh{c.cs, th, true, c.smem, npt};
            sh.mg = c.mg;
            cand.push_back(sh);
            break;
        }
    }
    const int saved_steps = L.nsteps;
    const int saved_cs = L.tuned_cs, saved_npt = L.tuned_npt, saved_th = L.tuned_threads;
    const bool saved_mg = L.tuned_mg;
    const mlq_options saved_opt = ctx->opt;
    ctx->opt.cluster = 0;
    ctx->opt.threads = 0;
    L.nsteps = probe_steps;
    cudaEvent_t e0, e1;
    MLQ_CUDA(ctx, cudaEventCreate(&e0));
    MLQ_CUDA(ctx, cudaEventCreate(&e1));
    double best = 1e300;
    Shape pick = cand[0];
    int st = MLQ_OK;
    for (int pass = 0; pass < 2 && st == MLQ_OK; ++pass) {  // pass 0 warms up
        for (const Shape &c : cand) {
            L.tuned_cs = c.cs;
            L.tuned_npt = c.npt;
            L.tuned_threads = c.threads;
            L.tuned_mg = c.mg;
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { st = MLQ_ECUDA; break; }
            st = mlq_solve(ctx, level, S, xi, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
            if (st != MLQ_OK) break;
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (pass == 1 && ms < best) {
                best = ms;
                pick = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    L.nsteps = saved_steps;
    ctx->opt = saved_opt;
    if (st != MLQ_OK) {
        L.tuned_cs = saved_cs;
        L.tuned_npt = saved_npt;
        L.tuned_threads = saved_th;
        L.tuned_mg = saved_mg;
        return st;
    }
    L.tuned_cs = pick.cs;
    L.tuned_npt = pick.npt;
    L.tuned_threads = pick.threads;
    L.tuned_mg = pick.mg;
    ctx->generation++;
    if (cluster_out) *cluster_out = pick.cs;
    if (threads_out) *threads_out = pick.threads;
    if (ms_out) *ms_out = best;
    return MLQ_OK;
}

// ---------------------------------------------------------------------------
// Solve without allocating: scratch in a fixed device array (see mlq.h).
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MLQ_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (host code may
// not use the symbol itself as a pointer).  Looked up once per device.
int noalloc_scratch(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return MLQ_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MLQ_ECUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return MLQ_OK;
}

// A pointer the kernels on device `dev` may use: device memory of that
// device, or managed memory.  Memory of another GPU is refused: the kernels
// would reach it only through peer access, which the call does not set up.
bool on_device(const void *p, int dev)
{
    if (!p) return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" {

int mlq_solve_noalloc(int m, double dt, int32_t nsteps, const mlq_model *model, const mlq_options *opt, int K,
                      const double *phi, const double *theta_mean, const double *xi, int64_t S, const double *v0,
                      const double *w0, double *q, int32_t *status, int32_t *iters, void *cuda_stream)
{
    if (m < 2 || m > 8193 || !(dt > 0.0) || nsteps < 0 || K < 1 || K > kMaxK || S < 0 || S > 65535) return MLQ_EINVAL;
    if (!phi || !xi || !q) return MLQ_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MLQ_ECUDA;
    if (!on_device(phi, dev) || !on_device(theta_mean, dev) || !on_device(xi, dev) || !on_device(v0, dev) ||
        !on_device(w0, dev) || !on_device(q, dev) || !on_device(status, dev) || !on_device(iters, dev))
        return MLQ_EINVAL;
    mlq_model md;
    if (model) md = *model;
    else mlq_default_model(&md);
    mlq_options o;
    if (opt) o = *opt;
    else mlq_default_options(&o, MLQ_MIXED);
    if (o.precision != MLQ_MIXED || validate_options(&o) != MLQ_OK) return MLQ_EINVAL;
    if (S == 0) return MLQ_OK;
    const int64_t n = (int64_t)m * m, ne = 2 * (int64_t)(m - 1) * (m - 1);
    // scratch layout: cs2 | A64 | A32 | v | w (2) | b | q | iters | status
    const size_t sn = (size_t)S * n;
    size_t off = 0;
    auto put = [&](size_t bytes) {
        const size_t at = off;
        off += align_up(bytes, 256);
        return at;
    };
    const size_t o_cs2 = put((size_t)S * ne * 16), o_a64 = put(sn * mlq::kSlots2D * 8),
                 o_a32 = put(sn * mlq::kSlots2D * 4), o_v = put(sn * 8), o_w = put(2 * sn * 8), o_b = put(sn * 8),
                 o_it = put((size_t)S * 4), o_st = put((size_t)S * 4);
    if (off > MLQ_NOALLOC_SCRATCH_BYTES) return MLQ_ETOOBIG;
    void *base = nullptr;
    int st = noalloc_scratch(dev, &base);
    if (st != MLQ_OK) return st;
    char *sc = (char *)base;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // launch shape: the smallest cluster whose register-kernel layout fits
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return MLQ_ECUDA;
    int cs = 0, npt = 0, threads = 0;
    for (int c = 1; c <= 8 && c <= m && cs == 0; c *= 2) {
        const mlq::RegPlan rp = mlq::reg_plan(m, c);
        if (rp.total > smem_optin - 2048) continue;
        for (int k : kNpt) {
            int th = ((rp.nmax + k - 1) / k + 31) / 32 * 32;
            if (th < 32) th = 32;
            if (th > npt_max_threads(k)) continue;
            cs = c;
            npt = k;
            threads = th;
            break;
        }
    }
    if (cs == 0) return MLQ_ETOOBIG;
    const mlq::RegPlan rp = mlq::reg_plan(m, cs);

    double *cs2 = (double *)(sc + o_cs2);
    double *A64 = (double *)(sc + o_a64);
    float *A32 = (float *)(sc + o_a32);
    mlq::kl_synthesis_kernel<<<dim3((unsigned)((ne + 255) / 256), (unsigned)S), 256, 0, stream>>>(
        phi, theta_mean, xi, K, (int)ne, (int)S, cs2);
    if (cudaGetLastError() != cudaSuccess) return MLQ_ECUDA;
    const double h = 1.0 / (double)(m - 1);
    mlq::stencil_setup_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)S), 256, 0, stream>>>(
        cs2, m, h, dt, md.s_l, md.s_t, (int)S, A64, A32);
    if (cudaGetLastError() != cudaSuccess) return MLQ_ECUDA;
    mlq::SolveArgs<float> a{};
    a.m = m;
    a.n = (int)n;
    a.h2 = h * h;
    a.dt = dt;
    a.nsteps = nsteps;
    a.a = md.a;
    a.eps = md.eps;
    a.gam = md.gamma;
    a.rtol_out = o.rtol;
    a.rtol_in = o.rtol_inner;
    a.max_iter = o.max_iter;
    a.max_sweeps = o.max_sweeps;
    a.A64 = A64;
    a.Ai = A32;
    a.v = (double *)(sc + o_v);
    a.w = (double *)(sc + o_w);
    a.b = (double *)(sc + o_b);
    a.v0 = v0;
    a.w0 = v0 ? w0 : nullptr;
    a.radius2 = 0.01;
    a.S = (int)S;
    a.q = q;
    a.iters = iters ? iters : (int32_t *)(sc + o_it);
    a.status = status ? status : (int32_t *)(sc + o_st);
    if (launch_reg_any(cs, npt, a, (int)S, threads, (size_t)rp.total, stream) != cudaSuccess) {
        cudaGetLastError();
        return MLQ_ECUDA;
    }
    return MLQ_OK;
}

int mlq_launch_count(mlq_ctx *ctx, int64_t *count)
{
    if (!ctx || !count) return MLQ_EINVAL;
    *count = ctx->launches;
    return MLQ_OK;
}

int mlq_level_launch(mlq_ctx *ctx, int level, int *cluster, int *threads, int *resident)
{
    MLQ_GUARD(ctx);
    if (!ctx || !cluster || !threads || level < 0 || level >= kMaxLevels || !ctx->levels[level].defined)
        return MLQ_EINVAL;
    const Shape sh = choose_launch(ctx, ctx->levels[level]);
    *cluster = sh.cs;
    *threads = sh.threads;
    if (resident) *resident = sh.mg ? 3 : (sh.npt > 0 ? 2 : (sh.resident ? 1 : 0));
    return MLQ_OK;
}

const char *mlq_strerror(int s)
{
    switch (s) {
    case MLQ_OK: return "ok";
    case MLQ_EINVAL: return "invalid argument";
    case MLQ_ENOMEM: return "out of memory";
    case MLQ_ECUDA: return "CUDA runtime error";
    case MLQ_ENOTREADY: return "not ready";
    case MLQ_ETIMEOUT: return "timed out";
    case MLQ_EUNSUPPORTED: return "not supported by this build";
    case MLQ_ETOOBIG: return "request exceeds the fixed scratch of mlq_solve_noalloc (MLQ_NOALLOC_SCRATCH_BYTES)";
    default: return "unknown status";
    }
}

const char *mlq_last_cuda_error(mlq_ctx *ctx)
{
    return ctx ? ctx->cuda_error.c_str() : "";
}

}  // extern "C"

// ===========================================================================
// Serving (mlq_submit / mlq_poll): continuous batching of per-level Monte
// Carlo requests.  A worker thread of the context owns up to kServeLanes
// lanes (a stream, a device workspace, pinned host buffers); every idle lane
// takes the next chunk of the waiting requests of one level (the level of
// the oldest waiting request no lane is serving) as one batched solve, so
// batches of different levels run on the device at the same time, and a
// request that arrives while others run starts as soon as a lane frees up.
// A batch is admitted by device memory: its lane's workspace grows only if
// the free HBM (and the optional budget of mlq_serve_limits) covers it;
// otherwise it waits for running batches, and a batch that cannot fit even
// with every other lane idle and released is refused (MLQ_ENOMEM).
// ===========================================================================
constexpr int kServeLanes = 6;
constexpr size_t kServeReserve = (size_t)256 << 20;   // HBM left free for the rest of the process
constexpr double kServeShortWork = 1.0e9;              // DOF-steps below which a batch is short

struct ServeReq {
    uint64_t id = 0;
    int level = 0;
    int64_t samples = 0;
    double target = 0.0;
    int64_t chunk = 16;
    int K = 0;
    std::vector<double> xi;  // samples x K
    int64_t next = 0;        // first sample not yet solved
    std::vector<double> q;
    std::vector<int32_t> st;
    int64_t checked = 0;     // chunk boundaries below this were tested
    bool finished = false;
    bool in_flight = false;  // a lane holds its next chunk
    mlq_result res{};
    std::chrono::steady_clock::time_point t0;
};

struct ServePart {
    ServeReq *r;
    int64_t first, count;
};

struct ServeLane {
    cudaStream_t stream = nullptr;      // the stream of the running batch (one of the two below)
    cudaStream_t s_hi = nullptr, s_lo = nullptr;   // highest / lowest stream priority
    cudaEvent_t done = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    double *h_xi = nullptr, *h_q = nullptr;   // pinned: batch inputs and outputs
    int32_t *h_st = nullptr, *h_err = nullptr;
    int64_t h_cap = 0;                        // samples the pinned buffers hold (x K for xi)
    int h_K = 0;
    bool busy = false;
    int level = -1;
    int64_t S = 0;
    double t_start = 0.0;
    std::vector<ServePart> parts;
};

struct Server {
    std::mutex mu;
    std::condition_variable cv;
    std::map<uint64_t, std::unique_ptr<ServeReq>> reqs;
    std::deque<uint64_t> order;  // arrival order of unfinished requests
    uint64_t next_id = 1;
    bool stop = false;
    int lanes = 4;               // lanes in use (mlq_serve_limits)
    size_t budget = 0;           // bytes of lane workspaces (0: free HBM only)
    ServeLane lane[kServeLanes];
    std::chrono::steady_clock::time_point epoch = std::chrono::steady_clock::now();
    std::thread worker;
};

namespace {

constexpr int64_t kServeMaxDofs = int64_t(1) << 24;  // DOFs per batched solve
constexpr int64_t kServeMaxSamples = int64_t(1) << 20;

double serve_ms(const Server &sv)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - sv.epoch).count();
}

// mean and sqrt(V_n / n) of the first n values, in index order
void serve_stats(const ServeReq &r, int64_t n, double *mean, double *rmse)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) m += r.q[i];
    m /= (double)n;
    double v = 0.0;
    for (int64_t i = 0; i < n; ++i) v += (r.q[i] - m) * (r.q[i] - m);
    v = n > 1 ? v / (double)(n - 1) : 0.0;
    *mean = m;
    *rmse = n > 1 ? std::sqrt(v / (double)n) : INFINITY;
}

void serve_finish(ServeReq &r, int64_t n, int status)
{
    r.finished = true;
    r.res.status = status;
    r.res.samples_used = n;
    int32_t worst = 0;
    for (int64_t i = 0; i < n; ++i) worst = std::max(worst, r.st[i]);
    r.res.worst = worst;
    if (n > 0) serve_stats(r, n, &r.res.mean, &r.res.rmse);
    r.res.latency_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r.t0).count();
}

// after new results: test the chunk boundaries in order
void serve_check(ServeReq &r)
{
    while (!r.finished) {
        const int64_t b = std::min(r.checked + r.chunk, r.samples);
        if (b > r.next) return;
        r.checked = b;
        double mean, rmse;
        serve_stats(r, b, &mean, &rmse);
        if ((r.target > 0.0 && b >= 2 && rmse <= r.target) || b == r.samples) serve_finish(r, b, MLQ_OK);
    }
}

void serve_prune(Server &sv)
{
    for (auto i = sv.order.begin(); i != sv.order.end();)
        i = sv.reqs.at(*i)->finished ? sv.order.erase(i) : i + 1;
}

// the workspace a batch of S samples of `level` takes on a lane
size_t serve_batch_bytes(const mlq_ctx *ctx, int level, int64_t S)
{
    const Level &L = ctx->levels[level];
    return member_bytes(ctx, L, S) + align_up((size_t)S * L.K * 8, 256);
}

// Lane workspaces come from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync): a plain cudaFree would wait for every
// running batch of every lane before it returns.
void serve_release(ServeLane &ln)
{
    if (ln.ws) cudaFreeAsync(ln.ws, ln.stream);
    ln.ws = nullptr;
    ln.ws_bytes = 0;
}

// device memory a new workspace can take: free HBM plus what the pool holds
// unused (freed lane workspaces not yet returned)
size_t serve_free_bytes(int device)
{
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaMemPool_t pool;
    uint64_t rsv = 0, used = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &rsv) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && rsv > used)
        fr += (size_t)(rsv - used);
    cudaGetLastError();
    return fr;
}

// Grow the lane's workspace to `bytes` if the device memory allows it:
// 1 = ready, 0 = not now (too little free memory), -1 = CUDA error.
int serve_reserve(const mlq_ctx *ctx, Server &sv, ServeLane &ln, size_t bytes, cudaStream_t st)
{
    size_t held = 0;
    for (int k = 0; k < sv.lanes; ++k) held += sv.lane[k].ws_bytes;
    if (ln.ws_bytes >= bytes && (sv.budget == 0 || held <= sv.budget)) return 1;
    if (sv.budget > 0 && held - ln.ws_bytes + bytes > sv.budget) return 0;
    const size_t fr = serve_free_bytes(ctx->device);
    if (fr + ln.ws_bytes < bytes + kServeReserve) return 0;
    serve_release(ln);
    if (cudaMallocAsync(&ln.ws, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        ln.ws = nullptr;
        return 0;
    }
    ln.ws_bytes = bytes;
    return 1;
}

int serve_host_buffers(ServeLane &ln, int64_t S, int K)
{
    if (S <= ln.h_cap && K <= ln.h_K) return MLQ_OK;
    cudaFreeHost(ln.h_xi);
    cudaFreeHost(ln.h_q);
    cudaFreeHost(ln.h_st);
    ln.h_xi = nullptr;
    ln.h_q = nullptr;
    ln.h_st = nullptr;
    ln.h_cap = 0;
    // grown geometrically from 4096 samples: freeing pinned memory waits
    // for the device, so it should happen rarely
    const int64_t cap = std::max<int64_t>(std::max<int64_t>(S, 4096), 2 * ln.h_cap);
    const int kk = std::max(K, ln.h_K);
    if (cudaMallocHost(&ln.h_xi, sizeof(double) * cap * kk) != cudaSuccess ||
        cudaMallocHost(&ln.h_q, sizeof(double) * cap) != cudaSuccess ||
        cudaMallocHost(&ln.h_st, sizeof(int32_t) * cap) != cudaSuccess) {
        cudaGetLastError();
        return MLQ_ENOMEM;
    }
    ln.h_cap = cap;
    ln.h_K = (int)kk;
    return MLQ_OK;
}

// queue one batch on a lane: xi in, the member's kernels, Q and status out,
// the device error flag, then the lane's event
int serve_launch(mlq_ctx *ctx, ServeLane &ln, int level, int64_t S)
{
    const Level &L = ctx->levels[level];
    char *cur = (char *)ln.ws;
    Member mb;
    mb.level = level;
    mb.S = S;
    member_carve(ctx, L, mb, cur);
    double *d_xi = (double *)cur;
    MLQ_CUDA(ctx, cudaMemcpyAsync(d_xi, ln.h_xi, sizeof(double) * S * L.K, cudaMemcpyHostToDevice, ln.stream));
    mb.d_xi = d_xi;
    int st = launch_member(ctx, mb, ln.stream, -1, 0);
    if (st != MLQ_OK) return st;
    MLQ_CUDA(ctx, cudaMemcpyAsync(ln.h_q, mb.q, sizeof(double) * S, cudaMemcpyDeviceToHost, ln.stream));
    MLQ_CUDA(ctx, cudaMemcpyAsync(ln.h_st, mb.status, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, ln.stream));
    MLQ_CUDA(ctx, cudaMemcpyAsync(ln.h_err, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, ln.stream));
    MLQ_CUDA(ctx, cudaEventRecord(ln.done, ln.stream));
    return MLQ_OK;
}

// results of a finished lane into its requests
void serve_harvest(Server &sv, ServeLane &ln, int code)
{
    if (code == MLQ_OK && *ln.h_err) code = MLQ_ETIMEOUT;
    const double now = serve_ms(sv);
    int64_t off = 0;
    for (const ServePart &p : ln.parts) {
        ServeReq &r = *p.r;
        r.in_flight = false;
        r.res.batches++;
        if (r.res.batches == 1) r.res.first_ms = ln.t_start;
        r.res.last_ms = now;
        if (code != MLQ_OK) {
            serve_finish(r, 0, code);
        } else {
            std::copy(ln.h_q + off, ln.h_q + off + p.count, r.q.begin() + p.first);
            std::copy(ln.h_st + off, ln.h_st + off + p.count, r.st.begin() + p.first);
            r.next = p.first + p.count;
            serve_check(r);
        }
        off += p.count;
    }
    ln.parts.clear();
    ln.busy = false;
    ln.level = -1;
}

// The next batch for an idle lane: the oldest waiting request no lane is
// serving sets the level; every waiting request at that level adds its next
// chunk (or all its samples without a target), up to the batch caps.
int64_t serve_form(mlq_ctx *ctx, Server &sv, std::vector<ServePart> &parts, int *level_out)
{
    parts.clear();
    std::lock_guard<std::recursive_mutex> g(ctx->mu);   // the level table
    // requests whose level changed its KL table (K) or was dropped since
    // submission cannot be served with the xi they brought
    for (uint64_t id : sv.order) {
        ServeReq &r = *sv.reqs.at(id);
        if (!r.finished && !r.in_flight &&
            (check_level(ctx, r.level) != MLQ_OK || ctx->levels[r.level].K != r.K))
            serve_finish(r, 0, MLQ_EINVAL);
    }
    // one batch per level on the device at a time: a level that already runs
    // in a lane waits, so a long batch of a fine level cannot take every lane
    // from the short batches of the coarse ones
    auto running = [&](int l) {
        for (int k = 0; k < sv.lanes; ++k)
            if (sv.lane[k].busy && sv.lane[k].level == l) return true;
        return false;
    };
    int level = -1, K = 0;
    for (uint64_t id : sv.order) {
        const ServeReq &r = *sv.reqs.at(id);
        if (!r.finished && !r.in_flight && !running(r.level)) {
            level = r.level;
            K = r.K;
            break;
        }
    }
    if (level < 0) return 0;
    const int64_t n = ctx->levels[level].n;
    const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(65535, kServeMaxDofs / std::max<int64_t>(n, 1)));
    int64_t total = 0;
    for (uint64_t id : sv.order) {
        ServeReq &r = *sv.reqs.at(id);
        if (r.finished || r.in_flight || r.level != level || r.K != K) continue;
        int64_t take = r.target > 0.0 ? std::min(r.chunk, r.samples - r.next) : r.samples - r.next;
        take = std::min(take, cap - total);
        if (take <= 0) break;
        parts.push_back({&r, r.next, take});
        total += take;
    }
    *level_out = level;
    return total;
}

void serve_loop(mlq_ctx *ctx, Server *svp)
{
    Server &sv = *svp;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(sv.mu);
    std::vector<ServePart> parts;
    for (;;) {
        bool busy = false;
        for (int k = 0; k < sv.lanes; ++k) busy = busy || sv.lane[k].busy;
        if (sv.stop && !busy) return;
        if (busy) sv.cv.wait_for(lk, std::chrono::microseconds(100));
        else if (!sv.stop) sv.cv.wait(lk, [&] { return sv.stop || !sv.order.empty(); });
        // finished batches
        for (int k = 0; k < sv.lanes; ++k) {
            ServeLane &ln = sv.lane[k];
            if (!ln.busy) continue;
            const cudaError_t q = cudaEventQuery(ln.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            serve_harvest(sv, ln, q == cudaSuccess ? MLQ_OK : MLQ_ECUDA);
        }
        if (sv.stop) continue;   // drain the running batches, start no new one
        // new batches on idle lanes
        for (int k = 0; k < sv.lanes; ++k) {
            ServeLane &ln = sv.lane[k];
            if (ln.busy) continue;
            int level = -1;
            const int64_t S = serve_form(ctx, sv, parts, &level);
            if (S <= 0) break;
            int K = 0;
            size_t bytes = 0;
            cudaStream_t bst;
            {
                std::lock_guard<std::recursive_mutex> g(ctx->mu);
                const Level &Lv = ctx->levels[level];
                K = Lv.K;
                bytes = serve_batch_bytes(ctx, level, S);
                // short batches on the high-priority stream: their CTAs take
                // the SMs that free up before the CTAs of long batches (a fine
                // level's CTA holds its SM for its sample's whole horizon)
                bst = (double)S * Lv.n * Lv.nsteps < kServeShortWork ? ln.s_hi : ln.s_lo;
            }
            int code = serve_host_buffers(ln, S, K);
            int got = code == MLQ_OK ? serve_reserve(ctx, sv, ln, bytes, bst) : -1;
            if (got == 0) {
                bool others = false;
                for (int j = 0; j < sv.lanes; ++j) others = others || sv.lane[j].busy;
                if (others) break;   // wait for a running batch to free memory
                for (int j = 0; j < sv.lanes; ++j) serve_release(sv.lane[j]);
                got = serve_reserve(ctx, sv, ln, bytes, bst);
                if (got == 0) code = MLQ_ENOMEM;   // cannot fit even alone: refuse
            }
            if (got != 1 || code != MLQ_OK) {
                for (const ServePart &p : parts) serve_finish(*p.r, 0, code != MLQ_OK ? code : MLQ_ECUDA);
                serve_prune(sv);
                sv.cv.notify_all();
                continue;
            }
            int64_t off = 0;
            for (const ServePart &p : parts) {
                std::memcpy(ln.h_xi + off * K, p.r->xi.data() + p.first * K, sizeof(double) * p.count * K);
                p.r->in_flight = true;
                off += p.count;
            }
            ln.parts = parts;
            ln.level = level;
            ln.S = S;
            ln.t_start = serve_ms(sv);
            ln.stream = bst;
            {
                std::lock_guard<std::recursive_mutex> g(ctx->mu);
                code = serve_launch(ctx, ln, level, S);
            }
            ln.busy = true;
            if (code != MLQ_OK) {
                cudaStreamSynchronize(ln.stream);
                cudaGetLastError();
                serve_harvest(sv, ln, code);
            }
        }
        serve_prune(sv);
        sv.cv.notify_all();
    }
}

void serve_stop(mlq_ctx *ctx)
{
    Server *sv = ctx->server.load();
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (ServeLane &ln : sv->lane) {
        serve_release(ln);
        if (ln.s_lo) cudaStreamSynchronize(ln.s_lo);
        if (ln.s_hi) cudaStreamSynchronize(ln.s_hi);
        cudaFreeHost(ln.h_xi);
        cudaFreeHost(ln.h_q);
        cudaFreeHost(ln.h_st);
        cudaFreeHost(ln.h_err);
        if (ln.done) cudaEventDestroy(ln.done);
        if (ln.s_lo) cudaStreamDestroy(ln.s_lo);
        if (ln.s_hi) cudaStreamDestroy(ln.s_hi);
    }
    ctx->server.store(nullptr);
    delete sv;
}

// the server with its lanes' streams and events; null on failure
Server *serve_create(mlq_ctx *ctx)
{
    std::unique_ptr<Server> sv(new Server());
    if (cudaSetDevice(ctx->device) != cudaSuccess) return nullptr;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (ServeLane &ln : sv->lane) {
        if (cudaStreamCreateWithPriority(&ln.s_lo, cudaStreamNonBlocking, lo) != cudaSuccess ||
            cudaStreamCreateWithPriority(&ln.s_hi, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&ln.h_err, sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            for (ServeLane &l2 : sv->lane) {
                if (l2.done) cudaEventDestroy(l2.done);
                if (l2.s_lo) cudaStreamDestroy(l2.s_lo);
                if (l2.s_hi) cudaStreamDestroy(l2.s_hi);
                cudaFreeHost(l2.h_err);
            }
            return nullptr;
        }
        ln.stream = ln.s_lo;
        *ln.h_err = 0;
    }
    return sv.release();
}

}  // namespace

extern "C" {

int mlq_submit(mlq_ctx *ctx, const mlq_request *req, uint64_t *ticket)
try {
    if (!ctx || !req || !ticket || !req->xi) return MLQ_EINVAL;
    const int64_t chunk = req->chunk > 0 ? req->chunk : 16;
    if ((chunk & (chunk - 1)) != 0 || req->samples < 1 || req->samples > kServeMaxSamples) return MLQ_EINVAL;
    auto r = std::make_unique<ServeReq>();
    {
        MLQ_GUARD(ctx);
        if (check_level(ctx, req->level) != MLQ_OK || ctx->levels[req->level].K < 1) return MLQ_EINVAL;
        r->K = ctx->levels[req->level].K;
        if (!ctx->server.load()) {
            Server *sv = serve_create(ctx);
            if (!sv) return MLQ_ECUDA;
            sv->lanes = ctx->serve_lanes;
            sv->budget = ctx->serve_budget;
            sv->worker = std::thread(serve_loop, ctx, sv);
            ctx->server.store(sv);
        }
    }
    r->level = req->level;
    r->samples = req->samples;
    r->target = req->target_rmse;
    r->chunk = chunk;
    r->xi.assign(req->xi, req->xi + (size_t)req->samples * r->K);
    r->q.assign(req->samples, 0.0);
    r->st.assign(req->samples, 0);
    r->t0 = std::chrono::steady_clock::now();
    Server &sv = *ctx->server.load();
    {
        std::lock_guard<std::mutex> lk(sv.mu);
        r->id = sv.next_id++;
        *ticket = r->id;
        sv.order.push_back(r->id);
        sv.reqs[r->id] = std::move(r);
    }
    sv.cv.notify_all();
    return MLQ_OK;
} catch (const std::bad_alloc &) {
    return MLQ_ENOMEM;
} catch (...) {  // thread creation
    return MLQ_ECUDA;
}

int mlq_serve_limits(mlq_ctx *ctx, int lanes, size_t max_bytes)
{
    if (!ctx || lanes < 1 || lanes > kServeLanes) return MLQ_EINVAL;
    {
        MLQ_GUARD(ctx);
        ctx->serve_lanes = lanes;
        ctx->serve_budget = max_bytes;
    }
    // the worker takes the server's lock before the context's: never hold
    // the context's lock here
    if (Server *sv = ctx->server.load()) {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (int k = lanes; k < kServeLanes; ++k)
            if (sv->lane[k].busy) return MLQ_ENOTREADY;   // shrink once those batches are done
        for (int k = lanes; k < kServeLanes; ++k) serve_release(sv->lane[k]);
        // idle lanes give their workspaces back: the next batch on each is
        // admitted against the new budget
        for (int k = 0; k < lanes; ++k)
            if (!sv->lane[k].busy) serve_release(sv->lane[k]);
        sv->lanes = lanes;
        sv->budget = max_bytes;
        sv->cv.notify_all();
    }
    return MLQ_OK;
}

int mlq_poll(mlq_ctx *ctx, uint64_t ticket, mlq_result *out)
{
    Server *svp = ctx ? ctx->server.load() : nullptr;
    if (!out || !svp) return MLQ_EINVAL;
    Server &sv = *svp;
    std::lock_guard<std::mutex> lk(sv.mu);
    auto i = sv.reqs.find(ticket);
    if (i == sv.reqs.end()) return MLQ_EINVAL;
    if (!i->second->finished) return MLQ_ENOTREADY;
    *out = i->second->res;
    sv.reqs.erase(i);
    return MLQ_OK;
}

}  // extern "C"
