#!/usr/bin/env python
"""Benchmark: multilevel Monte Carlo for the stochastic monodomain equation.

Workload (one "step" = one complete MLMC estimate, every level's fine and
coarse members):
  unit square, nested P1 triangulations on 17^2, 33^2, 65^2, 129^2, 257^2
  nodes; dt_l = 0.1 * 2^-l over T = 10 (100 ... 1600 time blocks);
  4096 / 1024 / 256 / 64 / 16 samples per level; FitzHugh-Nagumo kinetics
  (s_l 1, s_t 0.2, a 0.1, eps 0.01, gamma 0.5); initial quarter disc of
  radius 0.1; fibre angle = Gaussian KL field, 16 modes of
  0.09 exp(-|x-y|^2/0.04) on the finest mesh; xi ~ N(0,1) from Philox,
  seed = rank; QoI = integral of v at T.  Mixed precision (FP32 inner PCG
  preconditioned by a multigrid V-cycle, inside FP64 refinement to 1e-12), all
  levels running concurrently on prioritised streams, the whole estimate
  captured once into a CUDA graph and replayed (--no-graphs: eager launches).

Metric: DOF-steps/s (node x time block x sample, fine and coarse members
both counted); time-to-RMSE = wall time of one estimate.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mlq|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

LEVEL_M = [17, 33, 65, 129, 257]
LEVEL_N = [4096, 1024, 256, 64, 16]
K_MODES = 16
SIGMA2, ELL = 0.09, 0.04
T_END = 10.0
WORKLOAD = "MLMC 2D monodomain, 5 nested levels 17^2..257^2, N=4096/1024/256/64/16, K=16"
METRIC = "MLMC DOF-steps/s (time-to-RMSE of one estimate alongside)"
UNIT = "DOF-steps/s"
# Algorithmic bytes per DOF (2D) of the scope table's figure for this path: a
# matrix-free Jacobi-PCG as a memory-streaming solver moves them, each array
# read or written once per pass: 4 stencil coefficients 16 B + SpMV operand
# and result 8 B + vector updates 32 B = 56 B per CG iteration in FP32 (112 B
# in FP64), plus ~64 B per time block (reaction and load, FP64 refinement
# residual).  These bytes are the roofline's numerator whichever
# preconditioner runs; the multigrid kernel's own streaming count (one
# multigrid-PCG iteration: CG updates 44 B, pre-smoothing 12 B, residual 28 B,
# restriction 5 B, interpolation 9 B, post-smoothing 28 B, w = A u 24 B on the
# fine level, 150 B, plus a third of that V-cycle part for the coarse levels,
# 27 B: 176 B) is reported beside it.
BYTES_PER_DOF_ITER = {"mixed": 56.0, "fp64": 112.0}
BYTES_PER_DOF_STEP = 64.0
BYTES_PER_DOF_ITER_MG = 176.0


def level_dt(l):
    return 0.1 * 0.5 ** l


def level_steps(l):
    return int(round(T_END / level_dt(l)))


def dof_steps_per_estimate():
    tot = 0
    for l, N in enumerate(LEVEL_N):
        tot += N * LEVEL_M[l] ** 2 * level_steps(l)
        if l > 0:
            tot += N * LEVEL_M[l - 1] ** 2 * level_steps(l - 1)
    return tot


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def _oracle_setup():
    import oracle as O

    fine = O.mesh2d(LEVEL_M[-1])
    modes, _ = O.kl_build(fine, SIGMA2, ELL, K_MODES)
    meshes = [O.mesh2d(m) for m in LEVEL_M[:-1]] + [fine]
    phis = [O.centroid_table(fine, modes, mm) for mm in meshes]
    return O, meshes, phis


# Blocks every sampled member runs at least: the first blocks after the
# discontinuous initial state take several times the CG iterations of later
# ones, so a sample of only the first 1 % of a fine level's blocks (4 of 400
# at 65^2) understates the oracle's rate by up to 2x; from about 40 blocks on
# the sampled rate is within ~10-15 % of the whole horizon's (measured
# against a run of the whole workload).
ORACLE_MIN_BLOCKS = 40


def oracle_members(seed: int = 0, block_fraction: float = 0.01, full_levels=(0, 1)):
    """The members of the bounded oracle sample: every level pair l (fine
    member on mesh l, coarse member on mesh l-1, the same xi) takes its first
    S = min(N_l, max(16, host threads)) samples; pairs in `full_levels` run
    the whole horizon, the others max(ORACLE_MIN_BLOCKS, ceil(block_fraction
    * blocks)) blocks of each member (at most all).  A list of dicts (level,
    coarse, mesh level, samples, blocks, xi)."""
    from paper_2105_02007_gb300 import inputs

    import oracle as O

    threads = O.max_threads()
    out = []
    for l in range(len(LEVEL_M)):
        S = min(LEVEL_N[l], max(16, threads))
        xi = inputs.gaussian_xi(seed, l, 0, S, K_MODES)
        for coarse, lm in enumerate([l, l - 1] if l > 0 else [l]):
            full = level_steps(lm)
            steps = full if l in full_levels else min(full, max(ORACLE_MIN_BLOCKS,
                                                                int(np.ceil(block_fraction * full))))
            out.append(dict(level=l, coarse=coarse, mesh=lm, samples=S, blocks=steps, xi=xi))
    return out


def time_member(setup, mb):
    """Run one sampled member on every host thread; adds seconds, rate
    (DOF-steps/s) and q to the member's dict."""
    O, meshes, phis = setup
    lm = mb["mesh"]
    t0 = time.perf_counter()
    q, _, _ = O.solve_batch(meshes[lm], phis[lm], mb["xi"], level_dt(lm), mb["blocks"], nthreads=O.max_threads())
    el = time.perf_counter() - t0
    mb.update(seconds=el, rate=mb["samples"] * LEVEL_M[lm] ** 2 * mb["blocks"] / el, q=q)
    return mb


def whole_workload_seconds(rates):
    """Time of the whole workload extrapolated member by member: each
    member's DOF-steps over its measured rate; rates maps (level, coarse) to
    DOF-steps/s."""
    t = 0.0
    for l in range(len(LEVEL_M)):
        for coarse, lm in enumerate([l, l - 1] if l > 0 else [l]):
            t += LEVEL_N[l] * LEVEL_M[lm] ** 2 * level_steps(lm) / rates[(l, coarse)]
    return t


ORACLE_SAMPLE_DESC = ("every level pair l, first min(N_l, max(16, threads)) samples of both members; pairs 0,1 "
                      "over the whole horizon, the others over max(40, 1 %) of their time blocks; FP64 CSR "
                      "Jacobi-PCG, OpenMP over samples; whole-workload time extrapolated member by member from "
                      "the measured rates")


def oracle_sample(block_fraction: float = 0.01, seed: int = 0, setup=None):
    """The FP64 CPU oracle on a bounded sample of the workload (the members
    of oracle_members), each member timed once.  Returns a dict: value
    (DOF-steps/s of the whole workload, extrapolated), sample_value
    (DOF-steps/s over the sample), seconds, threads, members and a
    description."""
    setup = setup or _oracle_setup()
    members = [time_member(setup, mb) for mb in oracle_members(seed, block_fraction)]
    t_all = sum(m["seconds"] for m in members)
    dof_all = sum(m["samples"] * LEVEL_M[m["mesh"]] ** 2 * m["blocks"] for m in members)
    est = whole_workload_seconds({(m["level"], m["coarse"]): m["rate"] for m in members})
    return dict(value=dof_steps_per_estimate() / est, sample_value=dof_all / t_all, seconds=t_all,
                threads=setup[0].max_threads(), members=members, desc=ORACLE_SAMPLE_DESC, setup=setup)


def oracle_transient_ratio(setup, seed: int = 0):
    """How far the first blocks of a run misstate the oracle's rate: level 1
    (33 x 33 nodes, 200 blocks) with one sample per host thread over its
    first 4 blocks against the whole horizon (rate ratio)."""
    from paper_2105_02007_gb300 import inputs

    O, meshes, phis = setup
    threads = O.max_threads()
    xi = inputs.gaussian_xi(seed, 1, 0, max(16, threads), K_MODES)
    rates = []
    for steps in (4, level_steps(1)):
        t0 = time.perf_counter()
        O.solve_batch(meshes[1], phis[1], xi, level_dt(1), steps, nthreads=threads)
        rates.append(xi.shape[0] * LEVEL_M[1] ** 2 * steps / (time.perf_counter() - t0))
    return rates[0] / rates[1]


def oracle_single_thread(setup, block_fraction: float = 0.01, seed: int = 0):
    """The oracle on one host thread per level (the paper's work measure is
    single-thread time): one sample over the first ceil(block_fraction *
    steps) blocks of each level.  DOF-steps/s per level."""
    from paper_2105_02007_gb300 import inputs

    O, meshes, phis = setup
    out = []
    for l in range(len(LEVEL_M)):
        steps = max(1, int(np.ceil(block_fraction * level_steps(l))))
        xi = inputs.gaussian_xi(seed, l, 0, 1, K_MODES)
        t0 = time.perf_counter()
        O.solve_batch(meshes[l], phis[l], xi, level_dt(l), steps, nthreads=1)
        out.append(LEVEL_M[l] ** 2 * steps / (time.perf_counter() - t0))
    return out


def oracle_whole_workload():
    """The oracle's estimate and level variances of the whole workload (every
    sample of every level pair over the whole horizon, with its own KL
    tables), from the header of the fixture its script writes
    (tests/golden/mlmc_2d_5levels_oracle_y.txt); None without it."""
    path = os.path.join(ROOT, "tests", "golden", "mlmc_2d_5levels_oracle_y.txt")
    out = {}
    try:
        for line in open(path):
            w = line.split()
            if w and w[0] in ("estimate", "var", "rmse"):
                out[w[0]] = [float(x) for x in w[1:]]
            elif w and w[0] == "level":
                break
    except OSError:
        return None
    return out if "estimate" in out and "var" in out else None


def compare_with_oracle_whole(mean, var):
    """Relative differences of the library's estimate (and level variances,
    when given) from the oracle's whole-workload record; each side with the
    KL tables of its own builder."""
    ref = oracle_whole_workload()
    if ref is None:
        return None
    e = ref["estimate"][0]
    out = {"oracle_estimate": e, "estimate_rel": abs(mean - e) / abs(e),
           "source": "tests/golden/mlmc_2d_5levels_oracle_y.txt (FP64 oracle, every sample of every level pair "
                     "over the whole horizon; each side its own KL tables)"}
    if var is not None:
        out["var_rel_max"] = max(abs(a - b) / abs(b) for a, b in zip(var, ref["var"]))
    return out


def gpu_vs_oracle(mlq, prec, sample, phis):
    """The library on the oracle sample's members (same xi, same blocks, the
    oracle's mode tables phis as input): the largest relative difference of
    the per-sample QoI per member."""
    out = []
    with mlq.Context(0, prec) as ctx:
        for mb in sample["members"]:
            ctx.add_level(mb["mesh"], LEVEL_M[mb["mesh"]], level_dt(mb["mesh"]), mb["blocks"])
            ctx.set_kl(mb["mesh"], phis[mb["mesh"]])
            q = ctx.solve(mb["mesh"], mb["xi"])["q_fine"]
            out.append(float(np.max(np.abs(q - mb["q"]) / np.abs(mb["q"]))))
    return out


# ---------------------------------------------------------------------------
def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# device sources each slab kernel is compiled from (its translation unit and
# the headers holding its code)
KERNEL_SOURCES = {"slab_solve_mg_kernel": ("mlq_mg.cuh", "mlq_kernels.cuh", "mlq_reg_inst.cu"),
                  "slab_solve_reg_kernel": ("mlq_kernels.cuh", "mlq_reg_inst.cu"),
                  "slab_solve_kernel": ("mlq_kernels.cuh", "mlq_slab_inst.cu"),
                  "slab_solve_3d_kernel": ("mlq_3d.cuh", "mlq_3d_types.cuh", "mlq_groups.cuh", "mlq_kernels.cuh",
                                           "mlq_3d_inst.cu")}


def kernel_source_hash(kernel_key: str) -> str:
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2105_02007_gb300", "csrc")
    base = kernel_key.split("<")[0]
    files = KERNEL_SOURCES.get(base) or sorted(f for f in os.listdir(csrc) if f.endswith((".cuh", ".cu")))
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel_key: str, samples: int, steps: int):
    """DRAM bytes (read + write) per launch of `kernel_key`, from the committed
    ncu summary profiles/traffic.json, scaled from the captured cases to this
    launch; None if there is no capture for this kernel or the kernel sources
    changed since it was taken.  Two captures of one sample at different
    block counts give a per-sample set-up part and a per-block part
    (bytes = samples x (base + steps x per_block)); one capture scales by
    samples x blocks."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != kernel_source_hash(kernel_key) or not e.get("captures"):
        return None
    caps = sorted(e["captures"], key=lambda c: c["steps"])
    if len(caps) >= 2:
        a, b = caps[0], caps[-1]
        per_block = (b["dram_bytes"] / b["samples"] - a["dram_bytes"] / a["samples"]) / (b["steps"] - a["steps"])
        base = a["dram_bytes"] / a["samples"] - a["steps"] * per_block
        return samples * (base + steps * max(per_block, 0.0))
    c = caps[0]
    return c["dram_bytes"] * (samples * steps) / (c["samples"] * c["steps"])


def load_issue(kernel_key: str, member: dict):
    """Issue-rate ceiling of an on-chip kernel: warp instructions per DOF and
    CG iteration from an ncu capture (profiles/traffic.json, field "issue",
    same source hash), scaled to this launch and set against the SM array's
    issue rate (152 SMs x 4 schedulers x one warp instruction per cycle at
    the clock of the capture's kernel timing, taken as the maximum SM
    clock).  None without a current capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        e = json.load(open(path)).get(kernel_key)
    except Exception:
        return None
    if not e or e.get("source_hash") != kernel_source_hash(kernel_key) or "issue" not in e:
        return None
    iss = e["issue"]
    inst = iss["inst_per_dof_iter"] * member["cg_iterations"] * member["nodes"]
    sec = member["kernel_ms"] / 1000.0
    peak = iss["sms"] * 4 * iss["sm_mhz"] * 1e6
    return {"inst": inst, "achieved_inst_per_s": inst / sec, "peak_inst_per_s": peak, "frac": inst / sec / peak,
            "source": iss.get("source", "ncu smsp__inst_executed.sum")}


def roofline_3d(mlq, inputs, peaks):
    """The 3D member of the configuration's finest level (257 x 257 x 65 Kuhn
    nodes, 16 samples, one time block of dt = 0.05 / 8, mixed path with the
    multigrid preconditioner; K = 16 modes on the same mesh, the cost does not
    depend on K): its kernel's CUDA-event time after one warm-up solve, the
    algorithmic bytes of the streaming 3D solver (BYTES3D_* per DOF) over that
    time, and the DRAM traffic of an ncu capture when one is current."""
    level, S, steps, K = 3, 16, 1, 16
    dims = LEVEL3_DIMS[level]
    modes, _ = mlq.build_kl(dims, SIGMA2, ELL3, K)
    phi = mlq.centroid_table(dims, modes, dims)
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        ctx.add_level(level, dims, level3_dt(level), steps)
        ctx.set_kl(level, phi)
        ctx.set_profiling(True)
        xi = inputs.gaussian_xi(0, level, 0, S, K)
        ctx.solve(level, xi)
        ctx.solve(level, xi)
        prof = ctx.member_profile()[0]
    n = dims[0] * dims[1] * dims[2]
    it = prof["cg_iterations"]
    sec = prof["kernel_ms"] / 1e3
    algo = n * (it * BYTES3D_PER_DOF_ITER["mg"] + S * steps * BYTES3D_PER_DOF_STEP)
    hbm = peaks.get("hbm_gbs", 6800.0)
    coop = prof["cluster"] > 16   # CTAs per sample of a cooperative launch
    kname = "slab_solve_3d_kernel<float,GridGroup>" if coop else f"slab_solve_3d_kernel<float,ClusterGroup<{prof['cluster']}>>"
    traffic = load_traffic(kname, S, steps)
    out = {"bound": "hbm", "achieved": algo / sec / 1e9, "peak": hbm, "unit": "GB/s", "frac": algo / sec / 1e9 / hbm,
           "traffic": traffic, "kernel": kname, "kernel_ms": prof["kernel_ms"],
           "launch": f"{dims[0]}x{dims[1]}x{dims[2]} nodes, {S} samples, {steps} block, {it} CG iterations, "
                     + (f"{prof['cluster']} CTAs per sample in one cooperative launch" if coop
                        else f"cluster {prof['cluster']}"),
           "bytes": f"{BYTES3D_PER_DOF_ITER['mg']:.0f} B per DOF and CG iteration + {BYTES3D_PER_DOF_STEP:.0f} B "
                    "per DOF and block (the streaming 3D multigrid PCG, every array once per pass)",
           "dof_steps_per_s": n * S * steps / sec}
    if traffic:
        out["dram_gbs"] = traffic / sec / 1e9
        out["dram_frac"] = traffic / sec / 1e9 / hbm
    # the streaming count of a matrix-free 3D Jacobi-PCG iteration (88 B per
    # DOF: 48 B of fibre coefficients, 8 B product, 32 B update), which
    # leaves out the multigrid's passes
    jac = n * (it * 88.0 + S * steps * BYTES3D_PER_DOF_STEP)
    out["jacobi_pcg_count"] = {"bytes_per_dof_iter": 88.0, "achieved": jac / sec / 1e9, "frac": jac / sec / 1e9 / hbm}
    return out


def run_reference_full(setup):
    """The reference arm over the whole workload, once: every sample of every
    level pair over the whole horizon (about 3.7e9 DOF-steps: an hour or more
    of host time).  Prints the measured rate, the time of each member, and
    the oracle's estimate of eq. StandardML with its per-level variances."""
    from paper_2105_02007_gb300 import inputs

    O, meshes, phis = setup
    threads = O.max_threads()
    members, ys = [], []
    t_all = 0.0
    for l in range(len(LEVEL_M)):
        xi = inputs.gaussian_xi(0, l, 0, LEVEL_N[l], K_MODES)
        qs = []
        for coarse, lm in enumerate([l, l - 1] if l > 0 else [l]):
            t0 = time.perf_counter()
            q, it, st = O.solve_batch(meshes[lm], phis[lm], xi, level_dt(lm), level_steps(lm), nthreads=threads)
            el = time.perf_counter() - t0
            t_all += el
            qs.append(q)
            members.append(dict(level=l, coarse=coarse, mesh=LEVEL_M[lm], samples=LEVEL_N[l],
                                blocks=level_steps(lm), seconds=el, cg_iterations=int(np.sum(it)),
                                worst_status=int(np.max(st))))
            sys.stderr.write(f"[reference full] pair {l} {'coarse' if coarse else 'fine'}: {el:.1f} s\n")
            sys.stderr.flush()
        ys.append(qs[0] - qs[1] if l > 0 else qs[0])
    est, var, rmse = O.mlmc_estimate(ys)
    dof = dof_steps_per_estimate()
    desc = "the whole workload: every sample of every level pair over the whole horizon, FP64 CSR Jacobi-PCG, OpenMP over samples"
    line = {"impl": "reference", "metric": METRIC, "value": dof / t_all, "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 0, "ms_per_step": 1000.0 * t_all, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels": LEVEL_M, "samples": LEVEL_N, "K": K_MODES,
                       "dof_steps_per_step": dof, "precision": "fp64", "sample": desc},
            "cpu_baseline": {"value": dof / t_all, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": dof / t_all, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "estimate": est, "var_l": [float(v) for v in var], "rmse": rmse, "members": members}
    print(json.dumps(line), flush=True)
    return 0


def step_groups(M: int, K: int):
    """The members (indices 0 .. M-1) each of K timed steps runs: step j
    takes j, j + K, j + 2K, ... when K <= M, else member j mod M."""
    return [list(range(j, M, K)) if K <= M else [j % M] for j in range(K)]


def run_reference(args):
    """The reference arm: the oracle as it stands on the host cores.  The
    members of the bounded sample (oracle_members) are spread over the timed
    steps: with K timed steps, step j times the members j, j + K, j + 2K, ...
    of the list, or member j mod 9 when K > 9, so every member is timed at
    least once and the run costs about max(1, K / 9) passes over the sample
    (plus W warm-up steps, each one member).  The value is the whole
    workload's DOF-steps over its time extrapolated member by member from the
    mean measured rate of each member."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    setup = _oracle_setup()
    if args.full:
        return run_reference_full(setup)
    members = oracle_members(0)
    M, K = len(members), max(1, args.steps)
    for k in range(args.warmup):
        time_member(setup, dict(members[k % M]))
    rates, step_s = {}, []
    for idx in step_groups(M, K):
        group = [members[i] for i in idx]
        t = 0.0
        for mb in group:
            r = time_member(setup, dict(mb))
            rates.setdefault((mb["level"], mb["coarse"]), []).append(r["rate"])
            t += r["seconds"]
        step_s.append(t)
    rate = dof_steps_per_estimate() / whole_workload_seconds({k: sum(v) / len(v) for k, v in rates.items()})
    ms = 1000.0 * sum(step_s) / len(step_s)
    desc = ORACLE_SAMPLE_DESC + f"; the members spread over the {K} timed steps"
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels": LEVEL_M, "samples": LEVEL_N, "K": K_MODES,
                       "dof_steps_per_step": dof_steps_per_estimate(), "precision": "fp64", "sample": desc},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": setup[0].max_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_case(spec: str):
    """One member solve for profiling: --case level=L,samples=S,steps=N[,precision=mixed|fp64].
    Prints the slab-kernel time and iteration totals."""
    kv = dict(item.split("=") for item in spec.split(","))
    level = int(kv.get("level", 4))
    S = int(kv.get("samples", 1))
    steps = int(kv.get("steps", 4))
    prec_name = kv.get("precision", "mixed")
    from paper_2105_02007_gb300 import build, inputs

    build.build()
    from paper_2105_02007_gb300 import mlq

    prec = mlq.MLQ_MIXED if prec_name == "mixed" else mlq.MLQ_FP64
    modes, _ = mlq.build_kl(LEVEL_M[-1], SIGMA2, ELL, K_MODES)
    phi = mlq.centroid_table(LEVEL_M[-1], modes, LEVEL_M[level])
    with mlq.Context(0, prec) as ctx:
        ctx.add_level(level, LEVEL_M[level], level_dt(level), steps)
        ctx.set_kl(level, phi)
        ctx.set_profiling(True)
        xi = inputs.gaussian_xi(0, level, 0, S, K_MODES)
        res = ctx.solve(level, xi)
        prof = ctx.member_profile()[0]
    print(json.dumps({"case": spec, "kernel_ms": prof["kernel_ms"], "cg_iterations": prof["cg_iterations"],
                      "cluster": prof["cluster"], "threads": prof["threads"], "npt": prof["npt"],
                      "resident": prof["resident"], "q0": float(res["q_fine"][0])}))
    return 0


# 3D levels (Kuhn tetrahedra on [0,1]^2 x [0,0.25]): h_0 = 1/32 with 9 node
# planes, refined by halving; dt_0 = 0.05 halved per level, T = 10.
LEVEL3_DIMS = [(33, 33, 9), (65, 65, 17), (129, 129, 33), (257, 257, 65)]
ELL3 = 0.15 ** 2
# Algorithmic bytes per DOF of the 3D Jacobi-PCG (Chronopoulos-Gear) as a
# memory-streaming solver moves them, each array once per pass: update pass
# reads w s p x r u and 1/diag, writes s p x r u (48 B FP32); matvec pass
# reads 8 stencil slots and u, writes w (40 B FP32) -> 88 B per iteration;
# FP64 inner: 176 B.  Per block: reaction / w update (32 B), b = M y and
# r = b - A v (two FP64 15-point passes, stencil slots 64 B + vectors 28 B),
# one refinement residual (~90 B), v update (20 B) -> ~300 B.
# Multigrid (FP32): the CG update pass also forms the level-0 pre-smoothing
# (reads 1/diag, writes xa: 48 B with the updates) and the level-0
# post-smoothing (8 slots, xb, bb, 1/diag in, result out: 48 B) also forms
# (r, u); residual (8 slots, xa, bb in, rr out) 44 B, restriction 4 B,
# interpolation (xa, coarse in, xb out) 12 B; matvec 40 B; each coarser level
# an eighth of the V-cycle's 120 B (pre-smoothing 12 B there):
# 48 + 40 + 108 + 120 / 7 = 213 B.
BYTES3D_PER_DOF_ITER = {"mixed": 88.0, "fp64": 176.0, "mg": 213.0}
BYTES3D_PER_DOF_STEP = 300.0


def level3_dt(l):
    return 0.05 * 0.5 ** l


def run_case_mesh(spec: str):
    """One general-mesh solve on a synthetic left-ventricle shell:
    --case-mesh shell=M,samples=S,steps=N[,precision=fp64|mixed][,K=8][,cluster=C].
    Shell M is one of the four preset resolutions (~20k .. 1.3M nodes) with
    helix fibres; dt = 0.1 2^-M; a random KL table of K modes (scale 0.2).
    After a warm-up solve, times one solve on the host clock (the call
    returns when the results are on the host) and prints the time, CG
    iterations and time per iteration.  For profiling the general-mesh
    kernel with ncu."""
    kv = dict(item.split("=") for item in spec.split(",")) if spec else {}
    shell = int(kv.get("shell", 3))
    S = int(kv.get("samples", 1))
    steps = int(kv.get("steps", 1))
    K = int(kv.get("K", 8))
    prec_name = kv.get("precision", "fp64")
    cluster = int(kv.get("cluster", 0))
    from paper_2105_02007_gb300 import build, inputs
    from paper_2105_02007_gb300 import lv_inputs as LV

    build.build()
    from paper_2105_02007_gb300 import mlq

    prec = mlq.MLQ_MIXED if prec_name == "mixed" else mlq.MLQ_FP64
    xyz, conn, frames, alpha = LV.lv_level(shell)
    rng = np.random.default_rng(5)
    phi = rng.normal(scale=0.2, size=(conn.shape[0], K))
    v0, w0 = LV.stimulus(xyz, radius=0.4)
    xi = inputs.gaussian_xi(45, shell, 0, S, K)
    dt = 0.1 * 2.0 ** -shell
    with mlq.MeshLevel(xyz, conn, frames) as lvl:
        lvl.set_kl(phi, alpha)
        lvl.solve(xi, dt, steps, v0, w0, precision=prec, cluster=cluster)    # warm-up
        t0 = time.perf_counter()
        q, st, it = lvl.solve(xi, dt, steps, v0, w0, precision=prec, cluster=cluster)
        sec = time.perf_counter() - t0
    iters = int(np.sum(it))
    print(json.dumps({"case_mesh": spec, "nodes": int(xyz.shape[0]), "tets": int(conn.shape[0]), "seconds": sec,
                      "cg_iterations": iters, "us_per_iteration": 1e6 * sec / max(iters, 1),
                      "dof_steps_per_s": xyz.shape[0] * S * steps / sec, "q0": float(q[0]),
                      "status": [int(x) for x in st[:4]]}))
    return 0 if np.all(st == 0) else 1


def run_case3d(spec: str):
    """One 3D member solve: --case3d level=L,samples=S,steps=N[,precision=mixed|fp64][,K=16].
    KL modes of c = 0.09 exp(-|x-y|^2 / 0.15^2) on the level's own mesh.
    Prints time, DOF-steps/s, iterations and the algorithmic bandwidth
    against the measured HBM copy peak."""
    kv = dict(item.split("=") for item in spec.split(","))
    level = int(kv.get("level", 2))
    S = int(kv.get("samples", 4))
    steps = int(kv.get("steps", 2))
    K = int(kv.get("K", 16))
    prec_name = kv.get("precision", "mixed")
    from paper_2105_02007_gb300 import build, inputs

    build.build()
    from paper_2105_02007_gb300 import mlq

    prec = mlq.MLQ_MIXED if prec_name == "mixed" else mlq.MLQ_FP64
    precond = int(kv.get("precond", 1 if prec_name == "mixed" else 0))
    dims = LEVEL3_DIMS[level]
    modes, _ = mlq.build_kl(dims, SIGMA2, ELL3, K)
    phi = mlq.centroid_table(dims, modes, dims)
    with mlq.Context(0, prec, precond=precond) as ctx:
        ctx.add_level(level, dims, level3_dt(level), steps)
        ctx.set_kl(level, phi)
        ctx.set_profiling(True)
        xi = inputs.gaussian_xi(0, level, 0, S, K)
        ctx.solve(level, xi)    # warm-up
        res = ctx.solve(level, xi)
        prof = ctx.member_profile()[0]
    n = dims[0] * dims[1] * dims[2]
    it = prof["cg_iterations"]
    sec = prof["kernel_ms"] / 1e3
    per_it = BYTES3D_PER_DOF_ITER["mg" if (prec_name == "mixed" and precond == 1) else prec_name]
    algo = n * (it * per_it + S * steps * BYTES3D_PER_DOF_STEP)
    peaks = None
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = (peaks or {}).get("hbm_gbs", 6800.0)
    print(json.dumps({"case3d": spec, "dims": dims, "kernel_ms": prof["kernel_ms"], "cg_iterations": it,
                      "iterations_per_block": it / (S * steps), "cluster": prof["cluster"],
                      "threads": prof["threads"], "dof_steps_per_s": n * S * steps / sec,
                      "algorithmic_gbs": algo / sec / 1e9, "hbm_peak_gbs": hbm,
                      "frac": algo / sec / 1e9 / hbm, "q0": float(res["q_fine"][0]),
                      "status": [int(x) for x in res["status"][:4]]}))
    return 0


def run_c3(spec: str):
    """The 3D MLQMC estimator end to end: --c3 [T=10][,K=64][,L=3].
    Kuhn levels LEVEL3_DIMS[0..L], dt_l = 0.05 * 2^-l over [0, T]; KL modes of
    c = 0.09 exp(-|x-y|^2 / 0.15^2) on the finest mesh (K = 64 modes) transferred by
    the midpoint rule; per level 4^(L-l) lattice points (CBC generating
    vector, product weights lambda_k / lambda_1) x 16 random shifts, mapped to
    Gaussians; mlq_estimate over all levels (mixed path, multigrid).  Prints
    the DOF-steps/s of the timed estimate and the MLQMC estimate with its
    shift-based RMSE."""
    import time

    kv = dict(item.split("=") for item in spec.split(",")) if spec else {}
    T = float(kv.get("T", 10.0))
    K = int(kv.get("K", 64))
    L = int(kv.get("L", 3))
    R = 16
    from paper_2105_02007_gb300 import build, inputs

    build.build()
    from paper_2105_02007_gb300 import mlq

    dims = LEVEL3_DIMS[: L + 1]
    t0 = time.perf_counter()
    modes, lam = mlq.build_kl(dims[-1], SIGMA2, ELL3, K)
    phis = [mlq.centroid_table(dims[-1], modes, d) for d in dims]
    setup_s = time.perf_counter() - t0
    steps = [int(round(T / level3_dt(l))) for l in range(L + 1)]
    npts = [4 ** (L - l) for l in range(L + 1)]
    xis = [inputs.qmc_xi(0, l, npts[l], R, K, lam / lam[0]).reshape(-1, K) for l in range(L + 1)]
    ctx = mlq.Context(0, mlq.MLQ_MIXED)
    for l, d in enumerate(dims):
        ctx.add_level(l, d, level3_dt(l), steps[l])
        ctx.set_kl(l, phis[l])
    import torch

    torch.cuda.synchronize()
    t1 = time.perf_counter()
    mean, var, rmse_mc, ys = ctx.estimate(xis, return_y=True)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t1
    ctx.close()
    n = [d[0] * d[1] * d[2] for d in dims]
    dof = sum(len(xis[l]) * (n[l] * steps[l] + (n[l - 1] * steps[l - 1] if l > 0 else 0)) for l in range(L + 1))
    # MLQMC: per level the mean over the R shifts of the lattice means; the
    # error estimate from the spread over the shifts
    qmc_var = [float(np.var(np.asarray(y).reshape(R, -1).mean(axis=1), ddof=1) / R) for y in ys]
    print(json.dumps({"c3": spec or "T=10", "levels": [list(d) for d in dims], "steps": steps,
                      "solves": [len(x) for x in xis], "K": K, "seconds": sec, "dof_steps": dof,
                      "dof_steps_per_s": dof / sec, "estimate": mean, "rmse_qmc": float(sum(qmc_var) ** 0.5),
                      "host_kl_setup_s": setup_s}))
    return 0


def serve_stream(mlq, inputs, rate: float, nreq: int, lo: int, hi: int, chunk: int = 16, seed: int = 0):
    """A Poisson stream (exponential inter-arrival times, seed) of serving
    requests through mlq_submit / mlq_poll on one context: each picks a level
    uniformly in lo..hi, 1..256 samples, a target RMSE log-uniform in
    [1e-4, 1e-2] x |Qbar| (Qbar = 1.125e-3, the 2D estimate) and xi drawn with
    seed = request id.  Returns latency percentiles and served DOF-steps/s."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
    levels = rng.integers(lo, hi + 1, nreq)
    samples = rng.integers(1, 257, nreq)
    targets = 1.125e-3 * 10.0 ** rng.uniform(-4, -2, nreq)
    modes, _ = mlq.build_kl(LEVEL_M[-1], SIGMA2, ELL, K_MODES)
    ctx = mlq.Context(0, mlq.MLQ_MIXED)
    for l in range(lo, hi + 1):
        ctx.add_level(l, LEVEL_M[l], level_dt(l), level_steps(l))
        ctx.set_kl(l, mlq.centroid_table(LEVEL_M[-1], modes, LEVEL_M[l]))
    xis = [inputs.gaussian_xi(i, int(levels[i]), 0, int(samples[i]), K_MODES) for i in range(nreq)]
    # warm-up: one small request per level (kernel load, workspace)
    for l in range(lo, hi + 1):
        ctx.wait(ctx.submit(l, inputs.gaussian_xi(0, l, 0, 2, K_MODES), 0.0, 2))
    pending, done = {}, {}
    t0 = time.monotonic()
    i = 0
    while i < nreq or pending:
        now = time.monotonic() - t0
        while i < nreq and arrivals[i] <= now:
            pending[ctx.submit(int(levels[i]), xis[i], float(targets[i]), chunk)] = i
            i += 1
        for t in list(pending):
            r = ctx.poll(t)
            if r is not None:
                done[pending.pop(t)] = r
        time.sleep(0.001)
    wall = time.monotonic() - t0
    ctx.close()
    lat = np.array([done[k]["latency_ms"] for k in range(nreq)])
    used = np.array([done[k]["samples_used"] for k in range(nreq)])
    dof = sum(int(used[k]) * LEVEL_M[levels[k]] ** 2 * level_steps(int(levels[k])) for k in range(nreq))
    offered = rate * float(np.mean([LEVEL_M[l] ** 2 * level_steps(l) for l in range(lo, hi + 1)])) * 128.5
    by_level = {str(l): float(np.percentile(lat[levels == l], 50)) for l in range(lo, hi + 1) if np.any(levels == l)}
    return {"requests": nreq, "rate_per_s": rate, "levels": f"{lo}-{hi}", "completed": len(done),
            "status_ok": int(sum(done[k]["status"] == 0 for k in range(nreq))),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                           "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
            "p50_ms_by_level": by_level, "wall_s": wall, "samples_used_mean": float(used.mean()),
            "early_stop_fraction": float(np.mean(used < samples)),
            "served_dof_steps_per_s": dof / wall, "offered_dof_steps_per_s_at_full_samples": offered,
            "batches_mean": float(np.mean([done[k]["batches"] for k in range(nreq)]))}


def run_serve(spec: str):
    """Serving workload: --serve rate=R,requests=N[,levels=0-2][,chunk=16][,seed=0]
    (see serve_stream); prints its JSON record."""
    kv = dict(item.split("=") for item in spec.split(","))
    lo, hi = (int(x) for x in kv.get("levels", "0-2").split("-"))
    from paper_2105_02007_gb300 import build, inputs

    build.build()
    from paper_2105_02007_gb300 import mlq

    out = serve_stream(mlq, inputs, float(kv.get("rate", 50)), int(kv.get("requests", 200)), lo, hi,
                       int(kv.get("chunk", 16)), int(kv.get("seed", 0)))
    print(json.dumps({"serve": spec, **out}))
    return 0


def run_c5(spec: str):
    """The non-nested multilevel estimate on the synthetic left-ventricle
    shell: --c5 [T=0.1][,K=128][,N=1-4-16-64][,precision=fp64|mixed].
    Four unrelated tetrahedral shells (~20k, 80k, 320k, 1.3M nodes) with
    helix fibres (-60 to +60 deg transmurally) turned by a KL field of K modes
    of 0.09 exp(-|x-y|^2 / 0.25^2) built on the finest shell and moved to each
    shell's element centroids by point location on the device (P1
    interpolation between unrelated meshes); dt_m = 0.1 2^-m on shell m over
    [0, T]; eq. PimpedML
    with nested rules, term l on shell L-l at the first N_l Gaussian points.
    Prints the estimate, the time of each term's solve and DOF-steps/s.
    FP64 by default: the shells' thin elements make A ill-conditioned enough
    that FP32 inner solves stall before the FP64 residual reaches 1e-12."""
    kv = dict(item.split("=") for item in spec.split(",")) if spec else {}
    T = float(kv.get("T", 0.1))
    K = int(kv.get("K", 128))
    N = [int(x) for x in kv.get("N", "1-4-16-64").split("-")]
    prec_name = kv.get("precision", "fp64")
    from paper_2105_02007_gb300 import build, inputs
    from paper_2105_02007_gb300 import lv_inputs as LV

    build.build()
    import torch

    from paper_2105_02007_gb300 import mlq

    prec = mlq.MLQ_MIXED if prec_name == "mixed" else mlq.MLQ_FP64
    L = len(N) - 1

    def note(msg):
        sys.stderr.write(f"[c5 {time.strftime('%H:%M:%S')}] {msg}\n")
        sys.stderr.flush()

    t0 = time.perf_counter()
    shells = [LV.lv_level(m) for m in range(L + 1)]
    t_mesh = time.perf_counter() - t0
    note(f"meshes {t_mesh:.1f} s")
    xyzf, connf = shells[-1][0], shells[-1][1]
    t0 = time.perf_counter()
    modes, lam = mlq.build_kl_mesh(xyzf, connf, SIGMA2, 0.25 ** 2, K)
    t_kl = time.perf_counter() - t0
    note(f"KL {t_kl:.1f} s")
    t0 = time.perf_counter()
    cents = [sh[0][sh[1]].mean(axis=1) for sh in shells[:-1]]        # one device call for all coarse shells
    vals = mlq.p1_at_points(xyzf, connf, modes, np.concatenate(cents), device=True)
    cuts = np.cumsum([0] + [c.shape[0] for c in cents])
    phis = [vals[cuts[i]:cuts[i + 1]] for i in range(len(cents))]
    phis.append(modes[connf].mean(axis=1))
    t_transfer = time.perf_counter() - t0
    note(f"transfer {t_transfer:.1f} s")
    xi = inputs.gaussian_xi(0, 0, 0, max(N), K)
    F, per_term, dof = [], [], 0
    for l in range(L + 1):
        msh = L - l
        xyz, conn, frames, alpha = shells[msh]
        dt = 0.1 * 0.5 ** msh
        steps = int(round(T / dt))
        v0, w0 = LV.stimulus(xyz)
        with mlq.MeshLevel(xyz, conn, frames) as lvl:
            lvl.set_kl(phis[msh], alpha)
            lvl.solve(xi[:1], dt, 1, v0, w0, precision=prec)            # warm-up (kernel load)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            q, st, it = lvl.solve(xi[: N[l]], dt, steps, v0, w0, precision=prec)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t1
        F.append(q)
        note(f"term {l} shell {msh}: {N[l]} samples x {steps} blocks {sec:.2f} s, {np.mean(it) / steps:.0f} it/block")
        d = N[l] * xyz.shape[0] * steps
        dof += d
        per_term.append({"term": l, "shell": msh, "nodes": int(xyz.shape[0]), "tets": int(conn.shape[0]),
                         "samples": N[l], "blocks": steps, "seconds": sec, "dof_steps_per_s": d / sec,
                         "cg_iterations_per_block": float(np.mean(it)) / steps, "status_max": int(np.max(st))})
    est = mlq.pimped_ml_combine(F, N)
    total = sum(t["seconds"] for t in per_term)
    print(json.dumps({"c5": spec or "T=0.1", "K": K, "N": N, "precision": prec_name, "estimate": est,
                      "solve_seconds": total, "dof_steps": dof, "dof_steps_per_s": dof / total,
                      "terms": per_term, "host_setup_s": {"meshes": t_mesh, "kl": t_kl, "transfer": t_transfer}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mlq", choices=["mlq", "reference"])
    ap.add_argument("--full", action="store_true",
                    help="with --impl reference: the oracle over the whole workload, once (an hour or more)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed plain-FP64 estimates on the same xi (0: skip)")
    ap.add_argument("--jacobi-steps", type=int, default=1,
                    help="timed mixed-precision estimates with the Jacobi inner preconditioner, the FP64 path's "
                         "solver (0: skip)")
    ap.add_argument("--no-3d", action="store_true", help="skip the 257x257x65 3D member of the line")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving stream of the line")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--graphs", action="store_true", help="replay each estimate as a CUDA graph (the default)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="eager launches on the prioritised streams instead of the graph replay (measured 1414 ms "
                         "against 1390 ms per estimate)")
    ap.add_argument("--case", default=None, help="profile one member solve, e.g. level=4,samples=1,steps=4")
    ap.add_argument("--case3d", default=None, help="one 3D member solve, e.g. level=2,samples=8,steps=2")
    ap.add_argument("--case-mesh", default=None, nargs="?", const="",
                    help="one general-mesh solve on a ventricle shell, e.g. shell=3,samples=1,steps=1")
    ap.add_argument("--serve", default=None, help="serving stream, e.g. rate=50,requests=200,levels=0-2")
    ap.add_argument("--c5", default=None, nargs="?", const="",
                    help="non-nested estimate on the ventricle shells, e.g. T=0.1,K=128,N=1-4-16-64,precision=fp64")
    ap.add_argument("--c3", default=None, nargs="?", const="",
                    help="3D MLQMC estimate end to end, e.g. T=0.5,K=16,L=3")
    args = ap.parse_args()
    if args.case:
        return run_case(args.case)
    if args.case3d:
        return run_case3d(args.case3d)
    if args.case_mesh is not None:
        return run_case_mesh(args.case_mesh)
    if args.serve:
        return run_serve(args.serve)
    if args.c3 is not None:
        return run_c3(args.c3)
    if args.c5 is not None:
        return run_c5(args.c5)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2105_02007_gb300 import build, inputs

    build.build()
    from paper_2105_02007_gb300 import mlq

    stream = torch.cuda.Stream()
    prec = mlq.MLQ_MIXED if args.precision == "mixed" else mlq.MLQ_FP64
    modes, _ = mlq.build_kl(LEVEL_M[-1], SIGMA2, ELL, K_MODES)
    phis = [mlq.centroid_table(LEVEL_M[-1], modes, m) for m in LEVEL_M]

    def make_ctx(p):
        ctx = mlq.Context(local, p, stream=stream.cuda_stream, graphs=0 if args.no_graphs else 1)
        for l, m in enumerate(LEVEL_M):
            ctx.add_level(l, m, level_dt(l), level_steps(l))
            ctx.set_kl(l, phis[l])
        return ctx

    ctx = make_ctx(prec)
    # one allocation split over the ranks: rank r solves the contiguous sample
    # indices shard(N_l, r, W) of every level, with the xi of those indices
    from paper_2105_02007_gb300 import distributed as D

    shards = [D.shard(LEVEL_N[l], rank, world) for l in range(len(LEVEL_M))]
    if min(c for _, c in shards) < 2:
        raise SystemExit(f"{world} ranks leave fewer than 2 samples of a level per rank")
    xi_host = [inputs.gaussian_xi(0, l, f, c, K_MODES) for l, (f, c) in enumerate(shards)]
    xi_dev = [torch.from_numpy(x).to(f"cuda:{local}") for x in xi_host]
    xi_pin = [torch.from_numpy(x).pin_memory() for x in xi_host]
    torch.cuda.synchronize()
    # launch shapes: the library's autotuner on a 2-block probe of each level
    tuned = {}
    if prec == mlq.MLQ_MIXED and not args.no_autotune:
        for l in range(len(LEVEL_M)):
            tuned[l] = ctx.autotune(l, xi_dev[l], probe_steps=2)[:2]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{local}")

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- warm-up
    for _ in range(args.warmup):
        ctx.estimate(xi_dev)
    # ---- timed region: K estimates, inputs resident in HBM
    ctx.set_profiling(True)
    clocks = ClockSampler(local)
    launches0 = ctx.launch_count()
    step_ms, profiles, results = [], [], []
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()                                   # evict L2 between estimates
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = ctx.estimate(xi_dev)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            results.append(res)
            profiles.append(ctx.member_profile())
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = ctx.launch_count() - launches0
    ctx.set_profiling(False)
    ms = sum(step_ms) / len(step_ms)
    ms_all = ms
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_all = float(t.item())
    dof = dof_steps_per_estimate()          # the whole allocation, over all ranks
    dof_local = sum(c * (LEVEL_M[l] ** 2 * level_steps(l) + (LEVEL_M[l - 1] ** 2 * level_steps(l - 1) if l else 0))
                    for l, (_, c) in enumerate(shards))
    value = dof / (ms_all / 1000.0)

    # ---- end to end through the public call, host buffers (pinned) in and
    #      per-sample results out, copies inside the timed region
    e2e_vals = []
    h2d = sum(x.numel() * 8 for x in xi_pin)
    d2h = sum(c for _, c in shards) * 8 + 16 * len(LEVEL_N)
    e2e_y = None
    for _ in range(args.e2e_steps):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_y = ctx.estimate(xi_pin, return_y=True)[3]
        torch.cuda.synchronize()
        e2e_vals.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_vals) if e2e_vals else None
    combined = None
    if dist is not None:
        if e2e_s is not None:
            e2e_s = D.max_over_ranks(e2e_s)
        # the one exchange: every rank's Y_l to rank 0, merged in rank order
        ys = e2e_y if e2e_y is not None else ctx.estimate(xi_pin, return_y=True)[3]
        combined = D.combine_estimates(ys)

    # ---- roofline of the dominant kernel: the member launch that moves the
    #      most algorithmic bytes (members run concurrently, so each launch's
    #      event time includes sharing the GPU with the others)
    peaks = load_peaks()
    members = profiles[-1]
    pkey = args.precision

    def alg_bytes(d, per_iter=None):
        it = BYTES_PER_DOF_ITER[pkey] if per_iter is None else per_iter
        return d["nodes"] * (d["cg_iterations"] * it + d["samples"] * d["steps"] * BYTES_PER_DOF_STEP)

    k_dom = max(range(len(members)), key=lambda k: alg_bytes(members[k]))
    dom = members[k_dom]
    dom_ms = statistics.mean(p[k_dom]["kernel_ms"] for p in profiles)
    achieved = alg_bytes(dom) / (dom_ms / 1000.0) / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    if dom["resident"] == 3:
        kname = f"slab_solve_mg_kernel<{dom['cluster']},{dom.get('npt', 0)}>"
    elif dom["resident"] == 2:
        kname = f"slab_solve_reg_kernel<{dom['cluster']},{dom.get('npt', 0)}>"
    else:
        kname = (f"slab_solve_kernel<{'float' if pkey == 'mixed' else 'double'},{dom['cluster']},"
                 f"{'true' if dom['resident'] else 'false'}>")
    traffic = load_traffic(kname, dom["samples"], dom["steps"])
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "kernel": kname,
            "launch": f"level {dom['level']} {'coarse' if dom['coarse'] else 'fine'} member, "
                      f"{dom['samples']} samples x {dom['nodes']} nodes x {dom['steps']} blocks, "
                      f"{dom['cg_iterations']} CG iterations, cluster {dom['cluster']}",
            "kernel_ms": dom_ms, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks
            else "fallback 6800 GB/s",
            "bytes": f"{BYTES_PER_DOF_ITER[pkey]:.0f} B per DOF and CG iteration + {BYTES_PER_DOF_STEP:.0f} B per DOF "
                     "and block (matrix-free Jacobi-PCG streaming figure)",
            "note": "the kernel keeps its vectors in registers and shared memory (DRAM traffic far below the "
                    "algorithmic bytes); it is bound by on-chip latency and issue, not by HBM"
            if dom["resident"] else "algorithmic bytes over event time"}
    if dom["resident"] == 3:
        a_mg = alg_bytes(dom, BYTES_PER_DOF_ITER_MG) / (dom_ms / 1000.0) / 1e9
        roof["streaming_mg"] = {"bytes_per_dof_iter": BYTES_PER_DOF_ITER_MG, "achieved": a_mg, "frac": a_mg / hbm}
    issue = load_issue(kname, dom)
    if issue:
        roof["issue"] = issue
    mean, var, rmse = results[-1]
    y_mixed = e2e_y if e2e_y is not None else ctx.estimate(xi_dev, return_y=True)[3]

    # ---- comparators on the same inputs: the plain FP64 path (FP64 Jacobi-PCG)
    #      and the mixed path with the same Jacobi preconditioner (precision
    #      alone); errors of every QoI against the FP64 path
    def timed_estimates(c, k):
        c.estimate(xi_dev)
        t = []
        for _ in range(k):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.zero_()
                e0.record(stream)
                r = c.estimate(xi_dev, return_y=True)
                e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        return statistics.mean(t), r

    def qoi_errors(ref_mean, ref_y):
        return {"estimate_rel": abs(mean - ref_mean) / abs(ref_mean),
                "level_mean_rel": [float(abs(np.mean(a) - np.mean(b)) / abs(np.mean(b))) for a, b in zip(y_mixed, ref_y)],
                "per_sample_y_max_rel": [float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
                                         for a, b in zip(y_mixed, ref_y)]}

    fp64 = None
    if args.fp64_steps > 0 and prec == mlq.MLQ_MIXED and world == 1:
        c64 = make_ctx(mlq.MLQ_FP64)
        ms64, r64 = timed_estimates(c64, args.fp64_steps)
        c64.close()
        fp64 = {"value": dof / (ms64 / 1000.0), "unit": UNIT, "ms_per_step": ms64, "time_to_rmse_s": ms64 / 1000.0,
                "estimate": r64[0], "rmse": r64[2], "mixed_speedup": ms64 / ms,
                "solver": "FP64 Jacobi-PCG from v^n, ||r|| <= 1e-13 ||b|| (the oracle's algorithm)",
                "mixed_error_vs_fp64": qoi_errors(r64[0], r64[3])}
    jac = None
    if args.jacobi_steps > 0 and prec == mlq.MLQ_MIXED and world == 1:
        cj = make_ctx(mlq.MLQ_MIXED)
        cj.set_options(precond=0)
        msj, rj = timed_estimates(cj, args.jacobi_steps)
        cj.close()
        jac = {"value": dof / (msj / 1000.0), "unit": UNIT, "ms_per_step": msj, "estimate": rj[0],
               "solver": "mixed FP32/FP64 Jacobi-PCG (the FP64 path's preconditioner, FP32 inner)",
               "speedup_over_fp64": (fp64["ms_per_step"] / msj) if fp64 else None}

    # ---- one 3D member (257 x 257 x 65 Kuhn nodes, 16 samples, one block,
    #      mixed path, multigrid): algorithmic bytes over the kernel's time
    roof3d = None
    if not args.no_3d and prec == mlq.MLQ_MIXED and world == 1:
        roof3d = roofline_3d(mlq, inputs, peaks)

    # ---- serving: a Poisson stream at the configuration's rate (50/s) over
    #      levels 0-4, through mlq_submit / mlq_poll (continuous batching)
    serving = None
    if not args.no_serve and prec == mlq.MLQ_MIXED and world == 1:
        serving = serve_stream(mlq, inputs, 50.0, 100, 0, 4)

    cpu = None
    oracle_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = oracle_sample(0.01)
        ratio = oracle_transient_ratio(smp["setup"])
        single = oracle_single_thread(smp["setup"], 0.005)
        cpu = {"value": smp["value"], "unit": UNIT, "cores": smp["threads"], "kind": "oracle", "sample": smp["desc"],
               "seconds": smp["seconds"], "sample_value": smp["sample_value"],
               "first_blocks_over_whole_horizon_rate": ratio,
               "single_thread_dof_steps_per_s_by_level": single}
        oracle_err = {"members": [f"pair {m['level']} {'coarse' if m['coarse'] else 'fine'} ({m['blocks']} blocks)"
                                  for m in smp["members"]],
                      "per_sample_q_max_rel": gpu_vs_oracle(mlq, prec, smp, smp["setup"][2])}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32+f64" if pkey == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels": LEVEL_M, "samples": LEVEL_N, "K": K_MODES,
                       "dof_steps_per_step": dof, "dof_steps_per_rank": dof_local, "precision": pkey, "l2": "256 MiB buffer zeroed before each "
                       "timed estimate (inside the timed region, on the same stream)",
                       "parallelism": f"samples x{world} (contiguous index ranges of one allocation)",
                       "cuda_graph": not args.no_graphs,
                       "launch_shapes": {str(l): list(v) for l, v in tuned.items()}},
            "time_to_rmse_s": ms_all / 1000.0, "estimate": mean, "rmse": rmse, "var_l": list(var),
            "e2e": {"value": dof / e2e_s if e2e_s else None, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": len(e2e_vals)},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "roofline_3d": roof3d,
            "cpu_baseline": cpu, "fp64": fp64, "mixed_jacobi": jac, "error_vs_oracle": oracle_err,
            "serving": serving,
            "estimate_all_ranks": None if combined is None else {"estimate": combined[0], "rmse": combined[2],
                                                                  "ranks": world},
            "vs_oracle_whole_workload": compare_with_oracle_whole(combined[0], None) if combined is not None
            else compare_with_oracle_whole(mean, list(var)),
            "members": [{k: d[k] for k in ("level", "coarse", "cluster", "threads", "npt", "resident", "samples",
                                            "kernel_ms", "start_ms", "end_ms", "cg_iterations")}
                        for d in members],
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
