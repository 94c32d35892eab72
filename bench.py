#!/usr/bin/env python
"""Benchmark of the twisted-mass DD-alphaAMG hot path on one GB300.

One step = the whole path of the paper's method on one batch of synthetic
input: load the gauge field (SU(3) check, link packing, clover term), the
adaptive setup (test vectors, P, D_c(delta mu)), and the FGMRES solve of
D(mu) x = b to a true relative residual of 1e-10 (FP64 outer iteration,
FP32 K-cycle of eq. (1)).  Fig. 1 of the paper also times setup + solve.

Workload (default): 16^3 x 32 lattice, U = exp(0.5 i H), c_sw = 1.5,
mu = 0.003, delta = 5, two levels, N_v = 20, 4^4 aggregates and SAP
blocks, 3 setup iterations (few right-hand sides), one Gaussian rhs, m0 from
inputs/m0_tuned.json (near-critical).  Inputs per step (gauge 75 MB, test
vectors 503 MB, rhs 25 MB in FP64) exceed the 129 MB L2, so no extra flush.

Output: one JSON line (rank 0).  ``value`` is seconds per step with inputs
resident in HBM; ``e2e`` the same through the C ABI with pinned host
buffers (host->device copies and the device->host read of x inside the
timed region).  ``roofline`` rates the dominant kernel class by its
algorithmic bytes per launch over its CUDA-event time, measured live during
the timed steps.  ``cpu_baseline`` times the FP64 numpy oracle on a bounded
sample of the same workload and scales it by the unit counts of the run.

``--impl reference`` times the oracle alone (the reference arm of this
method is the CPU oracle; there is no other implementation to install).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "16x16x16x32_2lvl_nv20": dict(
        L=(32, 16, 16, 16), eps=0.5, seed=1, c_sw=1.5, mu=0.003, delta=5.0, nv=20,
        agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), setup_iters=3, tol=1e-10, coarse_mma=1,
        m0_key="16x16x16x32_eps0.5_seed1"),
    "24x24x24x48_2lvl_nv24_12pt": dict(
        L=(48, 24, 24, 24), eps=0.5, seed=1, c_sw=1.5, mu=0.002, delta=5.0, nv=24,
        agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), setup_iters=5, tol=1e-10, nrhs=12, point=True, coarse_mma=1,
        m0_key="16x16x16x32_eps0.5_seed1"),  # same field strength; the critical mass is a bulk quantity
    "48x48x48x96_3lvl_nv24_28_12pt": dict(
        L=(96, 48, 48, 48), eps=0.6, seed=1, c_sw=1.57551, mu=0.0009, delta=5.0, nv=24,
        agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), setup_iters=3, tol=1e-10, nrhs=12, point=True,
        levels=3, nv2=28, agg2=(2, 2, 2, 2), sap_block1=(2, 2, 2, 2), coarse_setup_iters=3,
        restart=16, rhs_batch=1, coarse_mma=1, sap1_prec=2, m0_key="16x16x16x32_eps0.6_seed1_csw1.57551",
        device_inputs=True),
    "8x8x8x8_2lvl_nv8": dict(
        L=(8, 8, 8, 8), eps=0.5, seed=5, c_sw=1.5, mu=0.005, delta=5.0, nv=8,
        agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), setup_iters=3, tol=1e-10, m0=-0.4),
}
# learned preconditioner stage, trained on 8 seeded fields and tested on 4 held-out ones
LEARNED = dict(L=(16, 16, 16, 16), eps=0.5, c_sw=1.5, mu=0.003, delta=5.0, nv=20, agg=(4, 4, 4, 4),
               sap_block=(4, 4, 4, 4), setup_iters=3, tol=1e-10, m0_key="16x16x16x32_eps0.5_seed1",
               train_seeds=tuple(range(101, 109)), test_seeds=tuple(range(201, 205)), pairs_per_field=256,
               epochs=8, batch=32, lr=2e-3)
WORKLOADS["16x16x16x16_learned"] = dict(LEARNED)
DEFAULT_WORKLOAD = "16x16x16x32_2lvl_nv20"
COUNTS_FILE = os.path.join(ROOT, "profiles", "bench_unit_counts.json")


def ncu_traffic(wl_name: str, kind: str) -> float | None:
    """DRAM bytes per rhs unit of a kernel class from a committed ncu capture,
    or None if there is none or the kernel's source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(wl_name, {}).get(kind)
    if not rec:
        return None
    files = {"sap": ["sap.cu", "tm_stencil.cuh", "tm_internal.cuh"],
             "dslash_f32": ["dirac.cu", "tm_stencil.cuh", "tm_internal.cuh"],
             "dslash_f64": ["dirac.cu", "tm_stencil.cuh", "tm_internal.cuh"]}.get(kind)
    if not files:
        return None
    m = hashlib.sha256()
    for f in files:
        m.update(open(os.path.join(ROOT, "paper_1611_01034_gb300", "csrc", f), "rb").read())
    return rec["bytes_per_unit"] if m.hexdigest()[:16] == rec["source_sha256_16"] else None


def workload_m0(wl: dict) -> tuple[float, str]:
    if "m0" in wl:
        return wl["m0"], "fixed"
    path = os.path.join(ROOT, "inputs", "m0_tuned.json")
    table = json.load(open(path))
    return float(table[wl["m0_key"]]["m0"]), "inputs/m0_tuned.json"


# ---------------------------------------------------------------------------
# algorithmic bytes per unit (one right-hand side) of each kernel class
# ---------------------------------------------------------------------------
def algorithmic_bytes(kind: str, wl: dict) -> tuple[float, float] | None:
    """(operator bytes per launch, vector bytes per rhs unit) a kernel class
    must move at minimum; a launch over u right-hand sides moves op + u * vec.

    dslash:   op = 4 links x 12 + clover 72 = 120 reals/site;
              vec = in + out spinor 48 reals/site
    sap:      one colour: op = links + clover on the colour's half (120 V/2);
              vec = x everywhere (24 V) + b and x-write on the half (48 V/2)
    restrict: op = P (24 N_v reals/site); vec = fine spinor 24 reals/site
    prolong:  op = P; vec = fine in/out 48 reals/site
    coarse_oe (one Schur application S = D_ee - D_eo D_oo^-1 D_oe, two
              launches): op = the 9 D_c blocks of every coarse site with the
              odd-site inverses in place of the odd self blocks, 9 (2N_v)^2
              complex per coarse site; vec = 2 coarse vectors
    coarse_build (one build of D_c): op = P, links and clover read once and
              D_c written; vec = 0
    """
    V = 1
    for n in wl["L"]:
        V *= n
    nv = wl["nv"]
    Vc = V
    for a in wl["agg"]:
        Vc //= a
    n = 2 * nv
    f = 4  # FP32 cycle
    if kind == "dslash_f64":
        return 120 * 8 * V, 48 * 8 * V
    if kind == "dslash_f32":
        return 120 * f * V, 48 * f * V
    if kind == "sap":
        return 120 * f * V / 2, (24 * V + 48 * V / 2) * f
    if kind == "restrict":
        return 24 * nv * f * V, 24 * f * V
    if kind == "prolong":
        return 24 * nv * f * V, 48 * f * V
    if kind == "coarse_oe":
        return 9 * n * n * 2 * f * Vc, 2 * n * 2 * f * Vc
    if kind == "coarse_build":
        return (24 * nv + 120) * f * V + 9 * n * n * 2 * f * Vc, 0.0
    return None


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle CPU baseline: per-unit costs on the full-size workload
# ---------------------------------------------------------------------------
def oracle_unit_costs(wl_name: str) -> dict:
    """Seconds per unit of each step component, timed on the oracle (FP64 numpy).

    Samples (full 16^3 x 32 lattice unless stated): the clover leaves of one
    ordered plane (x12 for the clover term); one D(mu) apply; one SAP colour
    half-sweep with 4 MR steps; one restriction and one prolongation with N_v
    vectors; the thin QR of all aggregates; 10 coarse odd-even GMRES steps on
    a coarse operator of the workload's shape; the local Galerkin build of
    D_c for N_v = 2 (scaled by columns x rows to N_v).
    """
    import numpy as np
    import inputs
    from oracle.dirac import Operator, clover_leaves
    from oracle.sap import SAP
    from oracle.coarse import Interpolation, CoarseOperator, OddEvenCoarse
    from oracle.krylov import gmres

    wl = WORKLOADS[wl_name]
    L, nv = wl["L"], wl["nv"]
    try:
        m0, _ = workload_m0(wl)
    except (OSError, KeyError):
        m0 = -0.5  # the unit costs do not depend on the value of m0
    U = inputs.gauge_field(L, wl["eps"], wl["seed"])
    out = {}
    t = time.perf_counter()
    clover_leaves(U, 0, 1)
    out["clover"] = 12 * (time.perf_counter() - t)
    op = Operator.__new__(Operator)
    op.U, op.L, op.m0, op.c_sw, op.mu, op.bc_t = U, tuple(L), m0, wl["c_sw"], wl["mu"], -1.0
    A = np.zeros(tuple(L) + (12, 12), dtype=np.complex128)
    A[...] = (m0 + 4) * np.eye(12)
    op.A = A
    psi = inputs.gaussian_spinor(L, 7)
    t = time.perf_counter()
    op.apply(psi)
    out["dslash_f64"] = time.perf_counter() - t
    sap = SAP(op, wl["sap_block"], n_mr=4)
    mask = sap.colour == 0
    t = time.perf_counter()
    r = psi - op.apply(psi)
    psi + sap.mr(r, mask) * mask[..., None, None]
    out["sap"] = time.perf_counter() - t
    tv = inputs.random_test_vectors(L, nv, 11)
    t = time.perf_counter()
    P = Interpolation(tv, wl["agg"])
    out["qr"] = time.perf_counter() - t
    t = time.perf_counter()
    rc = P.restrict(psi)
    out["restrict"] = time.perf_counter() - t
    t = time.perf_counter()
    psi + P.prolong(rc)
    out["prolong"] = time.perf_counter() - t
    rng = np.random.default_rng(0)
    n = 2 * nv
    blocks = (rng.standard_normal(P.Lc + (9, n, n)) + 1j * rng.standard_normal(P.Lc + (9, n, n))) * 0.05
    blocks[..., 0, :, :] += 4 * np.eye(n)
    oe = OddEvenCoarse(CoarseOperator(blocks, nv, wl["delta"] * wl["mu"]))
    t = time.perf_counter()
    gmres(oe.schur, oe.reduced_rhs(rc), tol=0.0, restart=30, maxit=10)
    out["coarse_iter"] = (time.perf_counter() - t) / 10
    # the build applies the operator to 2 N_v columns and projects each onto
    # 2 N_v rows: T(N_v) = 2 N_v alpha + 2 N_v^2 beta, fitted at N_v = 1 and 2
    tb = []
    for k in (1, 2):
        Pk = Interpolation(tv[:k], wl["agg"])
        t = time.perf_counter()
        CoarseOperator.build(op, Pk, 0.0)
        tb.append(time.perf_counter() - t)
    beta = max(0.0, (tb[1] - 2 * tb[0]) / 4)
    alpha = max(0.0, tb[0] / 2 - beta)
    out["coarse_build"] = 2 * nv * alpha + 2 * nv * nv * beta + out["qr"]
    return out


def oracle_seconds(costs: dict, counts: dict) -> float:
    """Oracle seconds per step = sum over components of count x unit cost."""
    return (counts["clover"] * costs["clover"]
            + counts["dslash_f64"] * costs["dslash_f64"]
            + counts["dslash_f32"] * costs["dslash_f64"]
            + counts["sap"] * costs["sap"]
            + counts["restrict"] * costs["restrict"]
            + counts["prolong"] * costs["prolong"]
            + counts["coarse_iter"] * costs["coarse_iter"]
            + counts["coarse_build"] * costs["coarse_build"])


def run_oracle_worker(wl_name: str) -> dict:
    """Time the unit costs in a fresh single-threaded process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    t0 = time.time()
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", wl_name],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle worker failed: " + r.stderr[-2000:])
    costs = json.loads(r.stdout.strip().splitlines()[-1])
    costs["_wall"] = time.time() - t0
    return costs


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
# multi-rank pieces of the contract (N GPUs = N independent replicas)
def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s replica: every rank solves its own system."""
    return base + rank


def max_over_ranks(sec: float, world: int, device) -> float:
    """The slowest rank's timed region (all ranks have passed a barrier)."""
    if world <= 1:
        return sec
    import torch
    import torch.distributed as dist
    t = torch.tensor([sec], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_step(sec_max: float, world: int, steps: int) -> float:
    """Whole-job value: the slowest rank's time over the steps all ranks ran."""
    return sec_max / (world * steps)


# ---------------------------------------------------------------------------
def main_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import inputs
    import paper_1611_01034_gb300 as tm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload]
    m0, m0_src = (args.m0, "command line") if args.m0 is not None else workload_m0(wl)
    L, nv, seed = wl["L"], wl["nv"], replica_seed(wl["seed"], rank)  # one independent replica per rank
    U = inputs.gauge_field(L, wl["eps"], seed)
    levels = wl.get("levels", 2)
    nrhs = wl.get("nrhs", 1)
    rb = args.rhs_batch or wl.get("rhs_batch", nrhs)  # right-hand sides per tm_solve call
    V = 1
    for n in L:
        V *= n
    Lc1 = tuple(L[d] // wl["agg"][d] for d in range(4))
    n_w = wl["nv2"] * (V // (wl["agg"][0] * wl["agg"][1] * wl["agg"][2] * wl["agg"][3])) * 2 * nv \
        if levels == 3 else 0
    if wl.get("device_inputs"):
        # the FP64 test vectors (tens of GB) are drawn on the device with a seeded
        # generator; the point sources are built there too; no host copies
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed + inputs.TV_SEED_OFFSET)
        tvd = torch.randn((nv * V * 12 + n_w,), dtype=torch.complex128, device="cuda", generator=gen)
        x0 = inputs.point_source_site(L, seed + inputs.RHS_SEED_OFFSET)
        site = ((x0[0] * L[1] + x0[1]) * L[2] + x0[2]) * L[3] + x0[3]
        bd = torch.zeros((12, V, 4, 3), dtype=torch.complex128, device="cuda")
        for k in range(12):
            bd[k, site, k // 3, k % 3] = 1.0
        Ud = torch.from_numpy(U).cuda()
        Uh = tvh = bh = xh = None
    else:
        tv = inputs.random_test_vectors(L, nv, seed + inputs.TV_SEED_OFFSET)
        if levels == 3:  # level-1 random vectors follow the fine ones
            w0 = inputs.random_coarse_vectors(Lc1, 2 * nv, wl["nv2"], seed + inputs.TV_SEED_OFFSET + 1)
            tv = np.concatenate([tv.ravel(), w0.ravel()])
        if wl.get("point"):
            b, _ = inputs.point_sources(L, seed + inputs.RHS_SEED_OFFSET)
        else:
            b = inputs.gaussian_spinor(L, seed + inputs.RHS_SEED_OFFSET)
        Ud, tvd, bd = (torch.from_numpy(a).cuda() for a in (U, tv, b))
        Uh, tvh, bh = (torch.from_numpy(a).pin_memory() for a in (U, tv, b))
        xh = torch.zeros(bh.shape, dtype=bh.dtype).pin_memory()
    xd = torch.zeros_like(bd)
    stream = torch.cuda.current_stream()
    extra = {k: wl[k] for k in ("nv2", "agg2", "sap_block1", "coarse_setup_iters", "restart", "sap1_prec")
             if k in wl}
    extra["coarse_mma"] = args.coarse_mma if args.coarse_mma is not None else wl.get("coarse_mma", 0)
    for kv in args.param or []:  # solver-parameter overrides, e.g. --param coarse_tol=0.02
        k, v = kv.split("=", 1)
        extra[k] = float(v) if "." in v or "e" in v else int(v)
    extra.setdefault("cycle_prec", tm.TM_F32)
    p = tm.params(L=L, m0=m0, c_sw=wl["c_sw"], mu=wl["mu"], delta=wl["delta"], nv=nv,
                  agg=wl["agg"], sap_block=wl["sap_block"], setup_iters=wl["setup_iters"],
                  max_rhs=rb, levels=levels, **extra)
    h = tm.tm_create(p, stream)
    infos = []

    def step(Ug, tvg, bg, xg):
        tm.tm_load_gauge(h, Ug)
        tm.tm_setup(h, tvg)
        xg.zero_()
        for r0 in range(0, nrhs, rb):
            st, info = tm.tm_solve(h, bg[r0:r0 + rb], xg[r0:r0 + rb], min(rb, nrhs - r0), wl["tol"])
            if st != tm.TM_OK:
                raise RuntimeError(f"solve failed: {tm.tm_status_string(st)}")
            infos.append(info.as_dict())

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(Ug, tvg, bg, xg, k, profile):
        barrier()
        torch.cuda.synchronize()
        if profile:
            tm.tm_profile(h, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            step(Ug, tvg, bg, xg)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / 1000.0, world, "cuda")

    for _ in range(max(0, args.warmup - 1)):
        step(Ud, tvd, bd, xd)
    # last warm-up step: time every kernel class once to find the dominant one
    tm.tm_profile(h, -1)
    step(Ud, tvd, bd, xd)
    prof_all = tm.tm_profile_read(h)
    tm.tm_profile(h, False)
    dom = max(prof_all, key=lambda k: prof_all[k]["ms"])
    kinds = [tm.tm_profile_name(k) for k in range(tm.tm_profile_kinds())]
    clocks = ClockSampler(local)
    clocks.start()
    infos.clear()
    # timed steps: every class counted, only the dominant class timed with events
    tm.tm_profile(h, 1 << kinds.index(dom))
    sec = timed(Ud, tvd, bd, xd, args.steps, profile=False)
    prof = tm.tm_profile_read(h)
    tm.tm_profile(h, False)
    clk = clocks.stop()
    step_infos = list(infos)
    del Ud, tvd, bd, xd  # the host-buffer run stages its own copies
    torch.cuda.empty_cache()
    sec_e2e = None
    h2d = d2h = 0
    if Uh is not None:
        # end-to-end through the C ABI with pinned host buffers
        step(Uh, tvh, bh, xh)
        sec_e2e = timed(Uh, tvh, bh, xh, args.steps, profile=False)
        h2d = (Uh.numel() + tvh.numel() + bh.numel() + xh.numel()) * 16
        d2h = xh.numel() * 16
    tm.tm_destroy(h)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    K = args.steps
    value = job_seconds_per_step(sec, world, K)
    # per-step unit counts (per rhs unit) from the profile
    per_step = {k: v["units"] / K for k, v in prof.items()}
    launches = sum(v["launches"] for v in prof.values())
    # kernel launches per profiled scope of a class (a Schur half is one
    # launch; a build scope is orthonormalisation + build + odd-site inverses)
    kernels_per_scope = {"coarse_oe": 2}
    roof = None
    model = algorithmic_bytes(dom, wl)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    if model is not None and prof[dom]["launches"]:
        # a build scope counts one unit (one D_c) whatever kernels it launches
        scopes = prof[dom]["units"] if dom == "coarse_build" else \
            prof[dom]["launches"] / kernels_per_scope.get(dom, 1)
        per_launch_bytes = model[0] + model[1] * prof[dom]["units"] / scopes
        avg_s = prof[dom]["ms"] / scopes / 1000.0
        achieved = per_launch_bytes / avg_s / 1e9
        tr = ncu_traffic(args.workload, dom)
        traffic = tr * prof[dom]["units"] / scopes if tr else None
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
                "bytes_per_launch": per_launch_bytes, "avg_launch_us": round(avg_s * 1e6, 2),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback"}
    tot_ms = sum(v["ms"] for v in prof_all.values())
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "share": round(v["ms"] / max(1e-12, tot_ms), 4)}
               for k, v in prof_all.items() if v["launches"]}
    # units per step; coarse_oe units count the odd-even Schur applications
    # (one per coarse GMRES step, plus the per-solve rhs/reconstruction)
    counts = {
        "clover": 1.0,
        "dslash_f64": per_step["dslash_f64"],
        "dslash_f32": per_step["dslash_f32"],
        "sap": per_step["sap"],
        "restrict": per_step["restrict"],
        "prolong": per_step["prolong"],
        "coarse_iter": per_step["coarse_oe"],
        "coarse_build": prof["coarse_build"]["units"] / K,
    }
    cpu = None
    if levels == 3:
        cpu = {"value": None, "unit": "s", "kind": "oracle",
               "note": "the oracle's per-unit cost model covers the two-level path only"}
    elif not args.no_cpu_baseline:
        try:
            costs = run_oracle_worker(args.workload)
            osec = oracle_seconds(costs, counts)
            cpu = {"value": round(osec, 2), "unit": "s", "cores": 1, "kind": "oracle",
                   "sample": ("FP64 numpy oracle, single thread, per-unit costs timed on the "
                              "full lattice (clover plane, D apply, SAP colour half-sweep, "
                              "restriction, prolongation, QR, 10 coarse GMRES steps, D_c build "
                              "at N_v=1,2 fitted as 2N_v a + 2N_v^2 b) x this run's unit counts per step"),
                   "sample_wall_s": round(costs["_wall"], 1),
                   "unit_costs_s": {k: round(v, 4) for k, v in costs.items() if not k.startswith("_")}}
        except Exception as e:  # report, do not hide
            cpu = {"value": None, "error": str(e)[:300]}
    scale = None
    if rank == 0 and world == 1 and not args.no_scale_kernels and args.workload == DEFAULT_WORKLOAD:
        try:
            scale = kernels_at_scale(peaks)
        except Exception as e:  # report, do not hide
            scale = {"error": str(e)[:300]}
    if args.write_counts:
        os.makedirs(os.path.dirname(COUNTS_FILE), exist_ok=True)
        json.dump({"workload": args.workload, "counts_per_step": counts,
                   "note": "unit counts per step of the hot path (algorithmic counts of this "
                           "method on this workload), used to scale the oracle's per-unit costs"},
                  open(COUNTS_FILE, "w"), indent=1)
    line = {
        "metric": "solve seconds to 1e-10 rel. residual; D(mu) HBM GB/s and D_c TFLOP/s vs peak",
        "value": round(value, 5),
        "unit": "s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(sec / K * 1000, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 outer / f32 cycle" if p.cycle_prec == tm.TM_F32 else "f64",
        "data": f"synthetic (seeded random SU(3) field U = exp({wl['eps']} i H); "
                + ("12 point sources)" if wl.get("point") else "Gaussian rhs)"),
        "config": {
            "workload": args.workload, "lattice_TZYX": list(L), "sites": V, "levels": levels,
            **({"nv2": wl["nv2"], "aggregate2": list(wl["agg2"]), "sap_block1": list(wl["sap_block1"]),
                "coarse_setup_iters": wl["coarse_setup_iters"]} if levels == 3 else {}),
            "restart": p.restart, "rhs_per_solve_call": rb, "coarse_mma": p.coarse_mma,
            "coarse_tol": p.coarse_tol, "post_smooth": p.post_smooth, "mr_iters": p.mr_iters,
            **({"sap1_prec": "f16" if p.sap1_prec == 2 else "f32"} if levels == 3 else {}),
            "nv": nv, "aggregate": list(wl["agg"]), "sap_block": list(wl["sap_block"]),
            "m0": m0, "m0_source": m0_src, "c_sw": wl["c_sw"], "mu": wl["mu"],
            "delta": wl["delta"], "setup_iters": wl["setup_iters"], "tol": wl["tol"], "nrhs": nrhs,
            "rhs": "12 spin-colour point sources" if wl.get("point") else "Gaussian",
            "step": f"load gauge + clover, adaptive setup, FGMRES solve ({nrhs} rhs, {rb} per call)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs per step > 129 MB L2 (no extra flush)",
        },
        "solve": {
            "outer_iters": [i["iters"] for i in step_infos],
            "coarse_iters": [i["coarse_iters"] for i in step_infos],
            "true_relres": max(i["true_relres"] for i in step_infos),
        },
        "e2e": ({"value": round(job_seconds_per_step(sec_e2e, world, K), 5), "unit": "s",
                 "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h} if sec_e2e is not None else
                {"value": None, "reason": "inputs generated on the device: pinned host copies of the FP64 "
                                          "test vectors would not fit the host memory twice"}),
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels_one_step": kernels,
        "kernels_at_scale": scale,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the oracle alone
# ---------------------------------------------------------------------------
def kernels_at_scale(peaks: dict) -> dict:
    """D(mu) applies and the tensor-core coarse Schur complement on a 24^3x48
    lattice (inputs larger than L2), timed with CUDA events on the library's
    stream: the D(mu) HBM GB/s and D_c TFLOP/s of the benchmark's metric."""
    import numpy as np
    import torch
    import inputs
    import paper_1611_01034_gb300 as tm

    L, nv = (48, 24, 24, 24), 24
    V = 1
    for n in L:
        V *= n
    stream = torch.cuda.current_stream()
    U = torch.from_numpy(inputs.gauge_field(L, 0.5, 1)).cuda()
    p = tm.params(L=L, m0=-0.41769, c_sw=1.5, mu=0.002, delta=5.0, nv=nv, agg=(4, 4, 4, 4),
                  sap_block=(4, 4, 4, 4), cycle_prec=tm.TM_F32, coarse_mma=1, max_rhs=12)
    h = tm.tm_create(p, stream)
    tm.tm_load_gauge(h, U)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {"lattice_TZYX": list(L)}

    def timed(fn, k=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k / 1e3

    for prec, name, esz in ((tm.TM_F32, "dslash_f32", 4), (tm.TM_F64, "dslash_f64", 8)):
        nb = tm.tm_field_bytes(h, 0, prec, 1)
        a = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        a.view(torch.float32 if esz == 4 else torch.float64).normal_()
        t = timed(lambda: tm.tm_apply(h, 0, prec, a, b, 1))
        byts = V * esz * (48 + 120)   # spinor in + out, 4 links x 12 reals, clover 72 reals per site
        out[name] = {"us": round(t * 1e6, 1), "algorithmic_bytes": byts, "achieved_gbs": round(byts / t / 1e9, 1),
                     "frac_of_measured_hbm": round(byts / t / 1e9 / hbm, 4),
                     "tflops": round(V * 2232 / t / 1e12, 3)}
        del a, b
    # 12-rhs odd-even coarse Schur complement on the tensor cores (TF32) after a setup from random vectors
    tv = torch.from_numpy(inputs.random_test_vectors(L, nv, 1 + inputs.TV_SEED_OFFSET)).cuda()
    tm.tm_setup_from_vectors(h, tv)
    del tv
    nh = V // 256 // 2
    n = 2 * nv
    R = 12
    v = torch.randn(R * nh * n * 2, device="cuda", dtype=torch.float32)
    y = torch.zeros_like(v)
    kinds = [tm.tm_profile_name(k) for k in range(tm.tm_profile_kinds())]
    for _ in range(3):
        tm.tm_schur(h, tm.TM_F32, v, y, R)
    tm.tm_profile(h, 1 << kinds.index("coarse_oe"))
    K = 20
    for _ in range(K):
        tm.tm_schur(h, tm.TM_F32, v, y, R)
    t = tm.tm_profile_read(h)["coarse_oe"]["ms"] / K / 1e3
    tm.tm_profile(h, False)
    flops = nh * 17 * n * n * 8 * R           # complex multiply-adds of the 17 blocks per site pair
    tiles = nh * 17 * (2 * n) * n * 4         # operator bytes read (FP32 tiles)
    out["coarse_schur_tf32"] = {"coarse_sites_per_parity": nh, "nv": nv, "nrhs": R, "us": round(t * 1e6, 1),
                                "tflops": round(flops / t / 1e12, 2), "operator_gbs": round(tiles / t / 1e9, 1),
                                "frac_of_measured_bf16": round(flops / t / 1e12 / float(peaks.get("bf16_tflops", 1900.0)), 4)}
    tm.tm_destroy(h)
    return out


def main_learned(args):
    """Train the learned layer on 8 fields, then solve on 4 held-out fields with
    no stage after the K-cycle, the learned layer (FP16 inference) and one SAP
    sweep in its place; report solve times (setup excluded) and iterations."""
    import numpy as np
    import torch
    import inputs
    import paper_1611_01034_gb300 as tm

    wl = WORKLOADS[args.workload]
    m0, m0_src = workload_m0(wl)
    L, nv = wl["L"], wl["nv"]
    stream = torch.cuda.current_stream()

    def handle(mode):
        p = tm.params(L=L, m0=m0, c_sw=wl["c_sw"], mu=wl["mu"], delta=wl["delta"], nv=nv, agg=wl["agg"],
                      sap_block=wl["sap_block"], setup_iters=wl["setup_iters"], cycle_prec=tm.TM_F32,
                      max_rhs=16, nn_mode=mode, nn_prec=tm.TM_F16)
        return tm.tm_create(p, stream)

    fr_bytes = None
    h = handle(0)
    rng = np.random.default_rng(7)
    w0 = 0.02 * (rng.standard_normal(2304) + 1j * rng.standard_normal(2304))
    tm.tm_nn_set_weights(h, w0)
    pairs = []
    t0 = time.time()
    npp = wl["pairs_per_field"]
    for seed in wl["train_seeds"]:
        U = torch.from_numpy(inputs.gauge_field(L, wl["eps"], seed)).cuda()
        tv = torch.from_numpy(inputs.random_test_vectors(L, nv, seed + inputs.TV_SEED_OFFSET)).cuda()
        tm.tm_load_gauge(h, U)
        tm.tm_setup(h, tv)
        fr_bytes = tm.tm_field_bytes(h, 0, tm.TM_F32, npp)
        r = torch.zeros(fr_bytes, dtype=torch.uint8, device="cuda")
        e = torch.zeros_like(r)
        e0 = torch.from_numpy(inputs.gaussian_spinor(L, seed + 3000, nrhs=npp)).cuda()
        tm.tm_nn_pairs(h, e0, r, e, npp)
        pairs.append((U, r, e))
        del tv, e0
    torch.cuda.synchronize()
    t_pairs = time.time() - t0
    t0 = time.time()
    losses = []
    for ep in range(wl["epochs"]):
        lsum = 0.0
        for U, r, e in pairs:
            tm.tm_load_gauge(h, U)
            lsum += float(tm.tm_nn_train(h, r, e, npp, 1, wl["batch"], wl["lr"])[0])
        losses.append(lsum / len(pairs))
    t_train = time.time() - t0
    w = tm.tm_nn_get_weights(h)
    tm.tm_destroy(h)
    del pairs
    torch.cuda.empty_cache()

    modes = {"plain": 0, "learned_fp16": 1, "sap_standin": 2}
    res = {k: {"solve_s": [], "iters": [], "true_relres": []} for k in modes}
    for seed in wl["test_seeds"]:
        U = torch.from_numpy(inputs.gauge_field(L, wl["eps"], seed)).cuda()
        tv = torch.from_numpy(inputs.random_test_vectors(L, nv, seed + inputs.TV_SEED_OFFSET)).cuda()
        b = torch.from_numpy(inputs.gaussian_spinor(L, seed + inputs.RHS_SEED_OFFSET)).cuda()
        for name, mode in modes.items():
            hh = handle(mode)
            tm.tm_load_gauge(hh, U)
            tm.tm_setup(hh, tv)
            tm.tm_nn_set_weights(hh, w)
            times = []
            for rep_ in range(1 + max(1, args.steps)):
                x = torch.zeros_like(b)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st, info = tm.tm_solve(hh, b, x, 1, wl["tol"])
                e1.record(stream)
                torch.cuda.synchronize()
                if st != tm.TM_OK:
                    raise RuntimeError(f"solve failed ({name}): {tm.tm_status_string(st)}")
                if rep_ > 0:
                    times.append(e0.elapsed_time(e1) / 1000.0)
            res[name]["solve_s"].append(statistics.median(times))
            res[name]["iters"].append(info.iters)
            res[name]["true_relres"].append(info.true_relres)
            tm.tm_destroy(hh)
    summary = {k: {"solve_s_mean": round(statistics.mean(v["solve_s"]), 5),
                   "iters": v["iters"], "max_true_relres": max(v["true_relres"])} for k, v in res.items()}
    print(json.dumps({
        "metric": "solve seconds to 1e-10 rel. residual (held-out fields, setup excluded)",
        "value": summary["learned_fp16"]["solve_s_mean"], "unit": "s", "n_gpus": 1,
        "higher_is_better": False, "dtype": "f64 outer / f32 cycle / f16 learned layer",
        "data": "synthetic (seeded random SU(3) fields U = exp(0.5 i H); Gaussian rhs)",
        "config": {"workload": args.workload, "lattice_TZYX": list(L), "m0": m0, "m0_source": m0_src,
                   "mu": wl["mu"], "delta": wl["delta"], "nv": nv, "train_fields": list(wl["train_seeds"]),
                   "test_fields": list(wl["test_seeds"]), "pairs": npp * len(wl["train_seeds"]),
                   "epochs": wl["epochs"], "batch": wl["batch"], "lr": wl["lr"]},
        "training": {"pairs_s": round(t_pairs, 2), "train_s": round(t_train, 2),
                     "loss_per_epoch": [round(l, 5) for l in losses]},
        "comparison": summary,
    }), flush=True)


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if not os.path.exists(COUNTS_FILE):
        print(json.dumps({"impl": "reference", "unavailable":
                          "no unit counts recorded (profiles/bench_unit_counts.json)"}))
        return
    counts = json.load(open(COUNTS_FILE))["counts_per_step"]
    times = []
    last = None
    for i in range(args.warmup + args.steps):
        costs = run_oracle_worker(args.workload)
        if i >= args.warmup:
            times.append(oracle_seconds(costs, counts))
        last = costs
    value = statistics.mean(times)
    print(json.dumps({
        "impl": "reference",
        "metric": "solve seconds to 1e-10 rel. residual; D(mu) HBM GB/s and D_c TFLOP/s vs peak",
        "value": round(value, 2), "unit": "s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": round(value, 2), "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": "per-unit oracle costs x recorded unit counts per step",
                         "unit_costs_s": {k: round(v, 4) for k, v in last.items() if not k.startswith("_")}},
        "e2e": {"value": round(value, 2), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--write-counts", action="store_true")
    ap.add_argument("--param", action="append", help="override a tm_params field: name=value")
    ap.add_argument("--rhs-batch", type=int, default=None, help="right-hand sides per tm_solve call")
    ap.add_argument("--no-scale-kernels", action="store_true",
                    help="skip the D(mu) and coarse Schur measurements on the 24^3x48 lattice")
    ap.add_argument("--oracle-worker", default=None)
    ap.add_argument("--m0", type=float, default=None, help="override the workload's tuned m0")
    ap.add_argument("--coarse-mma", type=int, default=None,
                    help="override the workload's coarse_mma (0 CUDA cores, 1..3 TF32 tensor-core products)")
    args = ap.parse_args()
    if args.oracle_worker:
        print(json.dumps(oracle_unit_costs(args.oracle_worker)))
        return
    if args.impl == "reference":
        main_reference(args)
    elif args.workload == "16x16x16x16_learned":
        main_learned(args)
    else:
        main_native(args)


if __name__ == "__main__":
    main()
