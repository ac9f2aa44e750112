// mlq_mesh_member.h -- a general-mesh level as a member of the library's
// solves and estimates (host side, implemented in mlq_mesh.cu): the device
// workspace of S samples carved from a caller-owned block, and the
// stream-ordered launch of the sample's KL synthesis, CSR assembly and block
// loop (no allocation, no host synchronisation: the calls can be captured
// into a CUDA graph).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mlq.h"
#include "mlq_points.cuh"

namespace mlq {

// launch shape of a member: G > 0 runs G CTAs per sample in one
// cooperative launch (every CTA resident), else one cluster of cs CTAs per
// sample
struct MeshShape {
    int cs = 1;
    int G = 0;
};

struct MeshWs {
    double *cs2 = nullptr, *aval = nullptr, *v = nullptr, *w = nullptr, *b = nullptr, *y = nullptr, *q = nullptr;
    float *a32 = nullptr;
    void *vec[7] = {};
    int32_t *iters = nullptr, *status = nullptr;
    unsigned *bar = nullptr;   // cooperative shape: per-sample barrier words
    double *part = nullptr;    // cooperative shape: per-CTA partial sums
};

int64_t mesh_nodes(const mlq_mesh *m);
int64_t mesh_elems(const mlq_mesh *m);
int mesh_modes(const mlq_mesh *m);

// launch shape for S samples: request 0 = chosen (a cooperative launch
// with G = min(CTAs resident / S, n / 2048) CTAs per sample when one
// cluster of 16 per sample leaves SMs idle and G > 16; else the cluster
// size), 1..16 = clusters of the power of two at or below it, > 16 = a
// cooperative launch of that many CTAs per sample (cs = 0 when they cannot
// all be resident)
MeshShape mesh_member_shape(const mlq_mesh *m, int64_t S, int request);
// bytes of the workspace of S samples in that shape (each piece 256-byte
// aligned)
size_t mesh_member_bytes(const mlq_mesh *m, bool mixed, int64_t S, const MeshShape &sh);
// the pieces of that workspace starting at base; base advances past it
MeshWs mesh_member_carve(const mlq_mesh *m, bool mixed, int64_t S, const MeshShape &sh, char *&base);
// enqueue the member on stream st: xi (S x K), v0 and w0 (n; w0 may be
// null) are device pointers; results in ws.q, ws.iters, ws.status.  setup:
// the KL synthesis and CSR assembly; solve: the block loop (one launch).
// err (device int) is set when a wait of the cooperative shape times out.
// points (may be null): point QoIs recorded after every block.
cudaError_t mesh_member_launch(const mlq_mesh *m, const mlq_model &model, const mlq_options &opt, double dt,
                               int nsteps, const double *d_v0, const double *d_w0, int64_t S, const double *d_xi,
                               const MeshWs &ws, const MeshShape &sh, int *err, cudaStream_t st, bool setup = true,
                               bool solve = true, const PointArgs *points = nullptr);

}  // namespace mlq
