#!/usr/bin/env python
"""Benchmark of the twisted-mass DD-alphaAMG hot path on one GB300.

One step = one FGMRES solve of D(mu) x = b (the K-cycle of eq. (1) as
preconditioner, Sec. 1) for one group of right-hand sides to a true relative
residual of 1e-10, with the setup (gauge field, clover term, adaptive setup
of P and the coarse operators) done once before the timed region and reported
separately, as the paper separates setup and solve costs (Fig. 1).

Default workload: 48^3 x 96, U = exp(0.6 i H), c_sw = 1.57551, mu = 0.0009,
delta = 5, three levels (N_v = 24 on 4^4 aggregates, then N_v2 = 28 on 2^4
level-1 aggregates; SAP blocks 4^4 with odd-even block solves as in Sec. 3,
3 post-smoothing sweeps, and 2^4 on level 1), 3 + 3 setup iterations, the 12
spin-colour point sources at one random site, solved in 2 steps of 6 (the
FGMRES(4) basis of 6 right-hand sides is what fits next to the setup data in
the 280 GB; restart 4 needs no more outer iterations than 8 or 16 here).  m0 from inputs/m0_tuned.json (near-critical).  Every field of
the step (2 GB per fine FP64 vector) is larger than the 129 MB L2, so no
flush is needed.

Output: one JSON line (rank 0).  ``value`` is seconds per step with the
inputs resident in HBM; ``e2e`` the same steps through the C ABI with pinned
host buffers (b, x0 host->device and x device->host inside the timed region),
cycling through the three groups of sources.  ``roofline`` rates the dominant
kernel class of the step by its algorithmic work per launch over its
CUDA-event time measured live during the timed steps.  ``cpu_baseline`` is
the FP64 numpy oracle: per-unit costs timed on the host (single thread, on
sample lattices, scaled per site) times the step's unit counts; its leg also
recomputes the true residual of one GPU solution with the oracle on the full
lattice, T-slab by T-slab over the host's cores.

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

TM_F32X2 = 4  # tm_params.outer_apply: FP32-pair products D(mu) z_k
PREC_NAMES = {0: "f64", 1: "f32", 2: "f16", 3: "bf16", 4: "f32x2"}

WORKLOADS = {
    "48x48x48x96_3lvl_nv24_28_12pt": dict(
        L=(96, 48, 48, 48), eps=0.6, seed=1, c_sw=1.57551, mu=0.0009, delta=5.0, nv=24,
        agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), setup_iters=3, tol=1e-10, nrhs=12, point=True,
        levels=3, nv2=28, agg2=(2, 2, 2, 2), sap_block1=(2, 2, 2, 2), coarse_setup_iters=3,
        restart=4, rhs_batch=6, coarse_mma=1, sap1_prec=2, outer_apply=TM_F32X2, block_oe=1,
        sap_prec=2, transfer_prec=2, post_smooth=3, coarse_tol=0.1,  # scanned: 4.91 -> 4.63 s per step
        m0_key="16x16x16x32_eps0.6_seed1_csw1.57551", device_inputs=True),
    "16x16x16x32_2lvl_nv20": dict(
        L=(32, 16, 16, 16), eps=0.5, seed=1, c_sw=1.5, mu=0.003, delta=5.0, nv=20,
        agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), setup_iters=3, tol=1e-10, coarse_mma=1,
        coarsest_steps=20,  # the launch-bound coarse solve as one CUDA graph: 50.9 -> 39.7 ms per step
        m0_key="16x16x16x32_eps0.5_seed1"),
    "24x24x24x48_2lvl_nv24_12pt": dict(
        L=(48, 24, 24, 24), eps=0.5, seed=1, c_sw=1.5, mu=0.002, delta=5.0, nv=24,
        agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), setup_iters=5, tol=1e-10, nrhs=12, point=True, coarse_mma=1,
        rhs_batch=12, m0_key="16x16x16x32_eps0.5_seed1"),  # same field strength; critical mass is a bulk quantity
    "8x8x8x8_2lvl_nv8": dict(
        L=(8, 8, 8, 8), eps=0.5, seed=5, c_sw=1.5, mu=0.005, delta=5.0, nv=8,
        agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), setup_iters=3, tol=1e-10, m0=-0.4),
}
# learned preconditioner stage, trained on 8 seeded fields and tested on 4 held-out ones
LEARNED = dict(L=(16, 16, 16, 16), eps=0.5, c_sw=1.5, mu=0.003, delta=5.0, nv=20, agg=(4, 4, 4, 4),
               sap_block=(4, 4, 4, 4), setup_iters=3, tol=1e-10, m0_key="16x16x16x32_eps0.5_seed1",
               train_seeds=tuple(range(101, 109)), test_seeds=tuple(range(201, 205)), pairs_per_field=1280,
               epochs=8, batch=32, lr=2e-3)
WORKLOADS["16x16x16x16_learned"] = dict(LEARNED)
DEFAULT_WORKLOAD = "48x48x48x96_3lvl_nv24_28_12pt"
COUNTS_FILE = os.path.join(ROOT, "profiles", "bench_unit_counts.json")
METRIC = "solve seconds to 1e-10 rel. residual; D(mu) HBM GB/s and D_c TFLOP/s vs peak"
# FP64 rate of GB300 from the nominal table: 1.25 TFLOP/s = 152 SMs x 2.07 GHz x 2 FMA/clk x 2
FP64_PEAK_TFLOPS = 1.25
# FP32 (CUDA cores): 152 SMs x 128 FMA/clk x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


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
    files = rec.get("files")
    if not files:
        return None
    m = hashlib.sha256()
    for f in files:
        m.update(open(os.path.join(ROOT, "paper_1611_01034_gb300", "csrc", f), "rb").read())
    return rec["bytes_per_unit"] if m.hexdigest()[:16] == rec["source_sha256_16"] else None


def workload_m0(wl: dict) -> tuple[float, str]:
    if "m0" in wl:
        return wl["m0"], "fixed"
    table = json.load(open(os.path.join(ROOT, "inputs", "m0_tuned.json")))
    return float(table[wl["m0_key"]]["m0"]), "inputs/m0_tuned.json"


def volumes(wl: dict) -> tuple[int, int, int]:
    """Sites of the fine, first coarse and (three levels) second coarse lattice."""
    V = 1
    for n in wl["L"]:
        V *= n
    a1 = 1
    for a in wl["agg"]:
        a1 *= a
    V1 = V // a1
    V2 = 0
    if wl.get("levels", 2) == 3:
        a2 = 1
        for a in wl["agg2"]:
            a2 *= a
        V2 = V1 // a2
    return V, V1, V2


# ---------------------------------------------------------------------------
# algorithmic work per launch of a kernel class (roofline numerators)
# ---------------------------------------------------------------------------
def sap_oe_flops_per_site(blk, n_mr: int) -> float:
    """Real flops of one odd-even SAP colour per site of the colour's half and
    right-hand side, counted from the algorithm (reading 5): a hop (spin
    projection, two SU(3) products, reconstruction) 168, the clover term with
    the twisted mass 600 and D_oo^-1 576 per site, the MR inner products and
    updates 192 per even site; H = the mean number of hops that stay inside a
    block (6 for 4^4 blocks).
      block residual r = b - D x on all sites:              1968
      Schur right-hand side (odd D_oo^-1, hops to even):    (576 + 168 H + 24) / 2
      each MR step (two half-hops, D_oo^-1, clover, MR):     (336 H + 576 + 600 + 192) / 2
      e_o = D_oo^-1 (r_o - D_oe e_e), x += e:                (168 H + 576) / 2 + 24"""
    H = sum(2.0 * (1.0 - 1.0 / b) for b in blk)
    return (1968 + 0.5 * (576 + 168 * H + 24) + n_mr * 0.5 * (336 * H + 576 + 600 + 192)
            + 0.5 * (168 * H + 576) + 24)


def roofline_model(kind: str, wl: dict, units: float, launches: float, outer: dict, peaks: dict) -> dict | None:
    """Bound, work per launch and peak of a kernel class.

    units / launches: right-hand-side units and kernel launches of the class
    in the timed steps; outer: {"iters": outer FGMRES iterations per rhs,
    "restart": m, "rhs": right-hand sides per step, "steps": timed steps}
    for the FP64 Arnoldi BLAS.  Bytes count every operator
    array once per launch and every vector once per right-hand side; flops
    count the arithmetic the definition needs.
      sap (one colour of a sweep): links + clover of the colour's half, x
        everywhere, b and the x update on the half: (120 V/2) op, (24 V + 48 V/2) vec reals;
        with odd-even block solves (also D_oo^-1 of the half's odd sites, 144 V/4
        reals) the FP32 flops of sap_oe_flops_per_site against the FP32 rate
      coarse_sap (level-1, one colour): the colour's D_c1 blocks once (9 n^2
        complex per site, FP16 copy with sap1_prec = TM_F16) + x everywhere,
        b and x on the half (FP32)
      restrict / prolong: P (24 N_v reals per site) + fine vectors
      level1 (D_c1 v): 9 n^2 complex per level-1 site + 2 vectors
      coarse_oe (one odd-even Schur application, 2 launches): 9 n^2 complex per
        coarsest site + 2 vectors
      dslash_f64: 2232 flop per site and rhs (FP64 ALU, 1344 B per site)
      dslash_f32x2: 672 B per site in FP32 input + FP64 output + FP32-pair
        links and clover (576 + 576 B per site once per launch): HBM bytes
      blas_fine: FP64 flops of the Arnoldi steps (CGS2: 2 k (k+1) complex
        multiply-adds per element in a cycle of k steps, plus norms, scaling
        and the solution update), FP64 ALU; in FP32-pair arithmetic
        (outer_apply = TM_F32X2) the vector bytes instead, HBM
    """
    V, V1, V2 = volumes(wl)
    nv = wl["nv"]
    n1 = 2 * nv
    f = 4  # FP32 cycle
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "recipe fallback 6.8 TB/s"
    if launches <= 0:
        return None
    per = units / launches  # rhs units per launch
    if kind == "sap":
        b = 120 * f * V / 2 + per * (24 * V + 48 * V / 2) * f
        if not wl.get("block_oe"):
            return {"bound": "hbm", "work": b, "unit": "GB/s", "peak": hbm, "peak_source": hbm_src}
        b += 144 * f * V / 4
        # odd-even block solves: about 20 flop per byte, above the FP32 ridge
        # (80.5 / 6.8 = 12 flop/B), so the FP32 rate is the roof
        fl = per * V / 2 * sap_oe_flops_per_site(wl["sap_block"], wl.get("mr_iters", 4))
        return {"bound": "alu", "work": fl / 1e3, "unit": "TFLOP/s", "peak": FP32_PEAK_TFLOPS, "scale": 1e9,
                "peak_source": "FP32 80.5 TFLOP/s (152 SMs x 128 FMA/clk x 2 x 2.07 GHz, nominal table)",
                "hbm_work": b, "hbm_peak": hbm}
    if kind == "coarse_sap":
        ob = 2 if wl.get("sap1_prec") == 2 else 4
        b = 9 * n1 * n1 * 2 * ob * V1 / 2 + per * (2 * n1 * V1 + 2 * 2 * n1 * V1 / 2) * f
        return {"bound": "hbm", "work": b, "unit": "GB/s", "peak": hbm, "peak_source": hbm_src}
    if kind == "restrict":
        return {"bound": "hbm", "work": 24 * nv * f * V + per * 24 * f * V, "unit": "GB/s", "peak": hbm,
                "peak_source": hbm_src}
    if kind == "prolong":
        return {"bound": "hbm", "work": 24 * nv * f * V + per * 48 * f * V, "unit": "GB/s", "peak": hbm,
                "peak_source": hbm_src}
    if kind == "level1":
        return {"bound": "hbm", "work": 9 * n1 * n1 * 2 * f * V1 + per * 2 * n1 * 2 * f * V1, "unit": "GB/s",
                "peak": hbm, "peak_source": hbm_src}
    if kind == "coarse_oe":
        n, Vc = (2 * wl["nv2"], V2) if wl.get("levels", 2) == 3 else (n1, V1)
        b = (9 * n * n * 2 * f * Vc + per * 2 * n * 2 * f * Vc) / 2  # two launches per application
        return {"bound": "hbm", "work": b, "unit": "GB/s", "peak": hbm, "peak_source": hbm_src}
    if kind == "dslash_f64":
        return {"bound": "alu", "work": 2232.0 * V * per / 1e3, "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                "peak_source": "FP64 1.25 TFLOP/s (152 SMs x 2.07 GHz x 2 FMA/clk x 2, nominal table)",
                "scale": 1e9}
    if kind == "dslash_f32x2":
        b = (576 + 576) * V + per * (96 + 192) * V
        return {"bound": "hbm", "work": b, "unit": "GB/s", "peak": hbm, "peak_source": hbm_src}
    if kind == "blas_fine" and wl.get("outer_apply") == TM_F32X2:
        # FP32-pair arithmetic on the FP64 vectors: HBM-bound; an Arnoldi step over
        # k basis vectors passes 3 k + 7 FP64 vectors, a cycle's solution update
        # reads its k FP32 z vectors and x twice (complex numbers: 12 V per rhs)
        m, it = outer["restart"], outer["iters"]
        vec = 0.0
        left = it
        while left > 0:
            kc = min(m, left)
            vec += sum(16 * (3 * k + 7) for k in range(1, kc + 1)) + 8 * kc + 32
            left -= kc
        total = vec * 12 * V * outer["rhs"] * outer["steps"]
        return {"bound": "hbm", "work": total / launches, "unit": "GB/s", "peak": hbm, "peak_source": hbm_src}
    if kind == "blas_fine":
        m, it = outer["restart"], outer["iters"]
        nrhs_total = outer["rhs"] * outer["steps"]  # right-hand sides solved in the timed steps
        flops_el = 0.0  # real flops per complex element of one rhs, whole solve
        left = it
        while left > 0:
            k = min(m, left)
            flops_el += 16 * k * (k + 1) + 4 * k + 2 * k + 8 * k + 6
            left -= k
        total = flops_el * 12 * V * nrhs_total
        return {"bound": "alu", "work": total / launches / 1e3, "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                "peak_source": "FP64 1.25 TFLOP/s (152 SMs x 2.07 GHz x 2 FMA/clk x 2, nominal table)",
                "scale": 1e9}
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
# oracle CPU baseline: per-unit costs on sample lattices, scaled per site
# ---------------------------------------------------------------------------
SAMPLE_L = (32, 16, 16, 16)


def oracle_unit_costs(wl_name: str) -> dict:
    """Seconds per unit and per site of each step component, timed on the
    FP64 numpy oracle in this (single-threaded) process.

    Fine units on a 16^3 x 32 sample lattice: one D(mu) apply; one SAP colour
    half-sweep (residual + MR steps on the colour's blocks, on the odd-even
    Schur complement when the workload uses it); one restriction
    and one prolongation with N_v vectors; one outer FGMRES(restart) iteration
    of CGS2 Arnoldi BLAS (trivial operator and preconditioner).  Two levels:
    ten odd-even coarse GMRES steps on a coarse operator of the workload's
    block size.  Three levels, on sample coarse lattices: a level-1 D_c1
    apply, a level-1 SAP colour, one P2 restriction or prolongation, a level-1
    FGMRES(coarse_restart) iteration of BLAS, ten odd-even GMRES steps on a
    coarsest operator of block size 2 N_v2.  Each cost is divided by the
    sample's sites; the workload's cost scales it by its own sites.
    """
    import numpy as np
    import inputs
    from oracle.dirac import Operator
    from oracle.sap import SAP
    from oracle.coarse import Interpolation, CoarseOperator, OddEvenCoarse
    from oracle.krylov import gmres

    wl = WORKLOADS[wl_name]
    nv, levels = wl["nv"], wl.get("levels", 2)
    try:
        m0, _ = workload_m0(wl)
    except (OSError, KeyError):
        m0 = -0.5  # the unit costs do not depend on the value of m0
    Ls = SAMPLE_L
    Vs = int(np.prod(Ls))
    U = inputs.gauge_field(Ls, wl["eps"], wl["seed"])
    out = {}
    op = Operator(U, m0, wl["c_sw"], wl["mu"])
    psi = inputs.gaussian_spinor(Ls, 7)
    t = time.perf_counter()
    op.apply(psi)
    out["dslash_site"] = (time.perf_counter() - t) / Vs
    oe = bool(wl.get("block_oe"))
    sap = SAP(op, wl["sap_block"], n_mr=4, block_oe=oe)
    mask = sap.colour == 0
    t = time.perf_counter()
    r = psi - op.apply(psi)
    psi + (sap.mr_oe(r, mask) if oe else sap.mr(r, mask)) * mask[..., None, None]
    out["sap_site"] = (time.perf_counter() - t) / Vs
    P = Interpolation(inputs.random_test_vectors(Ls, nv, 11), wl["agg"])
    t = time.perf_counter()
    rc = P.restrict(psi)
    out["restrict_site"] = (time.perf_counter() - t) / Vs
    t = time.perf_counter()
    psi + P.prolong(rc)
    out["prolong_site"] = (time.perf_counter() - t) / Vs
    rng = np.random.default_rng(0)
    m = wl.get("restart", 25)
    d = 1.0 + rng.random(psi.shape)
    nit = 2 * m
    t = time.perf_counter()
    gmres(lambda v: d * v, psi, tol=0.0, restart=m, maxit=nit, M=lambda v: v)
    out["outer_iter_site"] = (time.perf_counter() - t) / nit / Vs
    n = 2 * nv
    Lc1 = tuple(Ls[k] // wl["agg"][k] for k in range(4))
    V1s = int(np.prod(Lc1))

    def rand_blocks(Lc, nn, shift):
        b = (rng.standard_normal(Lc + (9, nn, nn)) + 1j * rng.standard_normal(Lc + (9, nn, nn))) * 0.05
        b[..., 0, :, :] += shift * np.eye(nn)
        return b

    if levels == 2:
        oe = OddEvenCoarse(CoarseOperator(rand_blocks(Lc1, n, 4.0), nv, wl["delta"] * wl["mu"]))
        t = time.perf_counter()
        gmres(oe.schur, oe.reduced_rhs(rc), tol=0.0, restart=30, maxit=10)
        out["coarse_iter_site"] = (time.perf_counter() - t) / 10 / V1s
        return out
    from oracle.multilevel import CoarseSAP, CoarseInterpolation
    nv2 = wl["nv2"]
    Dc1 = CoarseOperator(rand_blocks(Lc1, n, 4.0), nv, wl["mu"])
    v1 = rng.standard_normal(Lc1 + (n,)) + 1j * rng.standard_normal(Lc1 + (n,))
    t = time.perf_counter()
    Dc1.apply(v1)
    out["level1_apply_site"] = (time.perf_counter() - t) / V1s
    csap = CoarseSAP(Dc1, wl["sap_block1"], 4)
    cmask = csap.colour == 0
    t = time.perf_counter()
    r1 = v1 - Dc1.apply(v1)
    v1 + csap.mr(r1, cmask) * cmask[..., None]
    out["csap_site"] = (time.perf_counter() - t) / V1s
    w = rng.standard_normal((nv2,) + Lc1 + (n,)) + 1j * rng.standard_normal((nv2,) + Lc1 + (n,))
    P2 = CoarseInterpolation(w, wl["agg2"], nv)
    t = time.perf_counter()
    c2 = P2.restrict(v1)
    v1 + P2.prolong(c2)
    out["l1xfer_site"] = (time.perf_counter() - t) / 2 / V1s
    d1 = 1.0 + rng.random(v1.shape)
    m1 = 30
    t = time.perf_counter()
    gmres(lambda v: d1 * v, v1, tol=0.0, restart=m1, maxit=m1, M=lambda v: v)
    out["level1_iter_site"] = (time.perf_counter() - t) / m1 / V1s
    Lc2 = (4, 4, 4, 4)
    V2s = int(np.prod(Lc2))
    oe2 = OddEvenCoarse(CoarseOperator(rand_blocks(Lc2, 2 * nv2, 4.0), nv2, wl["delta"] * wl["mu"]))
    b2 = rng.standard_normal(Lc2 + (2 * nv2,)) + 1j * rng.standard_normal(Lc2 + (2 * nv2,))
    t = time.perf_counter()
    gmres(oe2.schur, oe2.reduced_rhs(b2), tol=0.0, restart=30, maxit=10)
    out["coarsest_iter_site"] = (time.perf_counter() - t) / 10 / V2s
    return out


def step_counts(prof: dict, steps: int, outer_iters: float, levels: int) -> dict:
    """Unit counts per step from the timed profile: D(mu) applies, SAP colour
    units, transfers, coarse steps; outer FGMRES iterations from the solve."""
    u = {k: v["units"] / steps for k, v in prof.items()}
    c = {"dslash": u.get("dslash_f64", 0) + u.get("dslash_f32x2", 0) + u.get("dslash_f32", 0),
         "sap": u.get("sap", 0), "restrict": u.get("restrict", 0), "prolong": u.get("prolong", 0),
         "outer_iter": outer_iters}
    if levels == 2:
        c["coarse_iter"] = u.get("coarse_oe", 0)
    else:
        c.update({"level1_apply": u.get("level1", 0), "csap": u.get("coarse_sap", 0),
                  "l1xfer": u.get("level1_transfer", 0), "coarsest_iter": u.get("coarse_oe", 0),
                  # each level-1 FGMRES step applies D_c1 once (restart residuals add a few)
                  "level1_iter": u.get("level1", 0)})
    return c


def oracle_seconds(costs: dict, counts: dict, wl: dict) -> float:
    """Oracle seconds per step = sum over components of count x per-site cost x sites."""
    V, V1, V2 = volumes(wl)
    s = (counts["dslash"] * costs["dslash_site"] * V + counts["sap"] * costs["sap_site"] * V
         + counts["restrict"] * costs["restrict_site"] * V + counts["prolong"] * costs["prolong_site"] * V
         + counts["outer_iter"] * costs["outer_iter_site"] * V)
    if "coarse_iter" in counts:
        return s + counts["coarse_iter"] * costs["coarse_iter_site"] * V1
    return s + (counts["level1_apply"] * costs["level1_apply_site"] * V1 + counts["csap"] * costs["csap_site"] * V1
                + counts["l1xfer"] * costs["l1xfer_site"] * V1 + counts["level1_iter"] * costs["level1_iter_site"] * V1
                + counts["coarsest_iter"] * costs["coarsest_iter_site"] * V2)


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


def _slab_worker(args):
    """One T-slab of the oracle's true residual (spawned process)."""
    from multiprocessing import shared_memory
    import numpy as np
    from oracle.slabs import slab_residual_norms
    names, shapes, m0, c_sw, mu, bc_t, t0, t1 = args
    shm = [shared_memory.SharedMemory(name=n) for n in names]
    try:
        U, x, b = (np.ndarray(sh, dtype=np.complex128, buffer=s.buf) for s, sh in zip(shm, shapes))
        return slab_residual_norms(U, x, b, m0, c_sw, mu, bc_t, t0, t1)
    finally:
        del U, x, b
        for s in shm:
            s.close()


def oracle_true_residual(U, x, b, m0, c_sw, mu, bc_t, workers: int) -> tuple[float, float]:
    """||b - D(mu) x|| / ||b|| by the oracle, slab by slab over `workers`
    spawned processes (the arrays in shared memory); returns (relres, seconds)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import numpy as np
    t0 = time.time()
    T = U.shape[0]
    shm, shapes = [], []
    try:
        for a in (U, x, b):
            s = shared_memory.SharedMemory(create=True, size=a.nbytes)
            np.ndarray(a.shape, dtype=np.complex128, buffer=s.buf)[...] = a
            shm.append(s)
            shapes.append(a.shape)
        slab = max(1, min(T // 2 - 1, -(-T // workers)))
        jobs = [([s.name for s in shm], shapes, m0, c_sw, mu, bc_t, t, min(T, t + slab)) for t in range(0, T, slab)]
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            res = pool.map(_slab_worker, jobs)
    finally:
        for s in shm:
            s.close()
            s.unlink()
    rr = sum(r[0] for r in res)
    bb = sum(r[1] for r in res)
    return float(np.sqrt(rr / bb)), time.time() - t0


# ---------------------------------------------------------------------------
# multi-rank pieces of the contract (N GPUs = N independent replicas)
# ---------------------------------------------------------------------------
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
# native arm
# ---------------------------------------------------------------------------
def point_source_group(L, x0, first: int, count: int, dtype_np=None, device=None):
    """Sources first..first+count-1 of the twelve spin-colour point sources at x0
    (source k = 3 s0 + c0), natural layout [count, T, Z, Y, X, 4, 3]."""
    import numpy as np
    V = int(np.prod(L))
    site = ((x0[0] * L[1] + x0[1]) * L[2] + x0[2]) * L[3] + x0[3]
    if device is not None:
        import torch
        b = torch.zeros((count, V, 4, 3), dtype=torch.complex128, device=device)
    else:
        b = np.zeros((count, V, 4, 3), dtype=np.complex128)
    for j in range(count):
        k = first + j
        b[j, site, k // 3, k % 3] = 1.0
    return b


def kernels_on_workload(h, tm, wl: dict, R: int, peaks: dict) -> dict:
    """D(mu) applies (FP32, FP64, FP32 pairs) and the coarse operators on the
    benchmark's own lattice with the setup just built, CUDA events on the
    library's stream: the D(mu) HBM GB/s and D_c TFLOP/s of the metric."""
    import torch
    V, V1, V2 = volumes(wl)
    stream = torch.cuda.current_stream()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {"lattice_TZYX": list(wl["L"])}

    def timed(fn, k=10):
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

    for pin, pout, name, byts in ((tm.TM_F32, tm.TM_F32, "dslash_f32", 168 * 4),
                                  (tm.TM_F64, tm.TM_F64, "dslash_f64", 168 * 8),
                                  (tm.TM_F32X2, tm.TM_F64, "dslash_f32x2", 96 + 192 + 576 + 576)):
        if pin == tm.TM_F32X2 and wl.get("outer_apply") != TM_F32X2:
            continue
        a = torch.zeros(tm.tm_field_bytes(h, 0, tm.TM_F32 if pin == tm.TM_F32X2 else pin, 1), dtype=torch.uint8,
                        device="cuda")
        b = torch.zeros(tm.tm_field_bytes(h, 0, pout, 1), dtype=torch.uint8, device="cuda")
        a.view(torch.float64 if pin == tm.TM_F64 else torch.float32).normal_()
        t = timed(lambda: tm.tm_apply(h, 0, pin, a, b, 1))
        out[name] = {"us": round(t * 1e6, 1), "algorithmic_bytes": byts * V,
                     "achieved_gbs": round(byts * V / t / 1e9, 1),
                     "frac_of_measured_hbm": round(byts * V / t / 1e9 / hbm, 4),
                     "tflops": round(V * 2232 / t / 1e12, 3)}
        del a, b
    # level-1 operator D_c1 with R right-hand sides (FP32 blocks)
    n1 = 2 * wl["nv"]
    nb = tm.tm_field_bytes(h, 1, tm.TM_F32, R)
    a = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    b = torch.zeros_like(a)
    a.view(torch.float32).normal_()
    t = timed(lambda: tm.tm_apply(h, 1, tm.TM_F32, a, b, R))
    fl = V1 * 9 * n1 * n1 * 8 * R
    out["level1_apply"] = {"nrhs": R, "us": round(t * 1e6, 1), "tflops": round(fl / t / 1e12, 3),
                           "operator_gbs": round(V1 * 9 * n1 * n1 * 8 / t / 1e9, 1)}
    del a, b
    torch.cuda.empty_cache()
    return out


def main_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import inputs
    import paper_1611_01034_gb300 as tm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    m0, m0_src = (args.m0, "command line") if args.m0 is not None else workload_m0(wl)
    L, nv, seed = wl["L"], wl["nv"], replica_seed(wl["seed"], rank)  # one independent replica per rank
    # host inputs first: the gauge generator's process pool is spawned before any CUDA call
    U = inputs.gauge_field(L, wl["eps"], seed, workers=min(16, os.cpu_count() or 1))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    levels = wl.get("levels", 2)
    nrhs = wl.get("nrhs", 1)
    R = args.rhs_batch or wl.get("rhs_batch", nrhs)  # right-hand sides per step
    groups = max(1, nrhs // R)
    V, V1, V2 = volumes(wl)
    n_w = wl["nv2"] * V1 * 2 * nv if levels == 3 else 0
    if wl.get("device_inputs"):
        # the FP64 test vectors (tens of GB) are drawn on the device with a seeded generator
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed + inputs.TV_SEED_OFFSET)
        tvd = torch.randn((nv * V * 12 + n_w,), dtype=torch.complex128, device="cuda", generator=gen)
    else:
        tv = inputs.random_test_vectors(L, nv, seed + inputs.TV_SEED_OFFSET)
        if levels == 3:  # level-1 random vectors follow the fine ones
            Lc1 = tuple(L[d] // wl["agg"][d] for d in range(4))
            w0 = inputs.random_coarse_vectors(Lc1, 2 * nv, wl["nv2"], seed + inputs.TV_SEED_OFFSET + 1)
            tv = np.concatenate([tv.ravel(), w0.ravel()])
        tvd = torch.from_numpy(tv).cuda()
        del tv
    x0 = inputs.point_source_site(L, seed + inputs.RHS_SEED_OFFSET) if wl.get("point") else None

    def host_group(g):
        if x0 is not None:
            return point_source_group(L, x0, g * R, R)
        return inputs.gaussian_spinor(L, seed + inputs.RHS_SEED_OFFSET + g, nrhs=R).reshape(R, V, 4, 3)

    stream = torch.cuda.current_stream()
    extra = {k: wl[k] for k in ("nv2", "agg2", "sap_block1", "coarse_setup_iters", "restart", "sap1_prec",
                                "outer_apply", "block_oe", "sap_prec", "transfer_prec", "coarsest_steps", "post_smooth",
                                "coarse_tol") if k in wl}
    extra["coarse_mma"] = args.coarse_mma if args.coarse_mma is not None else wl.get("coarse_mma", 0)
    for kv in args.param or []:  # solver-parameter overrides, e.g. --param coarse_tol=0.02
        k, v = kv.split("=", 1)
        extra[k] = float(v) if "." in v or "e" in v else int(v)
    extra.setdefault("cycle_prec", tm.TM_F32)
    p = tm.params(L=L, m0=m0, c_sw=wl["c_sw"], mu=wl["mu"], delta=wl["delta"], nv=nv,
                  agg=wl["agg"], sap_block=wl["sap_block"], setup_iters=wl["setup_iters"],
                  max_rhs=R, levels=levels, **extra)
    h = tm.tm_create(p, stream)
    kinds = [tm.tm_profile_name(k) for k in range(tm.tm_profile_kinds())]

    # ---- setup (once, outside the timed steps) ---------------------------------
    Ud = torch.from_numpy(U).cuda()
    torch.cuda.synchronize()
    tm.tm_profile(h, -1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tm.tm_load_gauge(h, Ud)
    tm.tm_setup(h, tvd)
    e1.record(stream)
    torch.cuda.synchronize()
    setup_s = e0.elapsed_time(e1) / 1000.0
    prof_setup = tm.tm_profile_read(h)
    tm.tm_profile(h, False)
    del Ud, tvd
    torch.cuda.empty_cache()

    # ---- device-resident steps ---------------------------------------------------
    bd = torch.from_numpy(host_group(0)).cuda()
    xd = torch.zeros_like(bd)
    infos = []

    def step(bg, xg):
        xg.zero_()
        st, info = tm.tm_solve(h, bg, xg, R, wl["tol"])
        if st != tm.TM_OK:
            raise RuntimeError(f"solve failed: {tm.tm_status_string(st)}: {tm.tm_last_error(h)}")
        infos.append(info.as_dict())

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(k, one_step):
        barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(k):
            one_step(i)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(t0.elapsed_time(t1) / 1000.0, world, "cuda")

    for _ in range(max(0, args.warmup - 1)):
        step(bd, xd)
    # last warm-up step: time every kernel class once to find the dominant one
    tm.tm_profile(h, -1)
    step(bd, xd)
    prof_all = tm.tm_profile_read(h)
    tm.tm_profile(h, False)
    dom = max(prof_all, key=lambda k: prof_all[k]["ms"])
    clocks = ClockSampler(local)
    clocks.start()
    infos.clear()
    # timed steps: every class counted, only the dominant class timed with events
    tm.tm_profile(h, 1 << kinds.index(dom))
    sec = timed(args.steps, lambda i: step(bd, xd))
    prof = tm.tm_profile_read(h)
    tm.tm_profile(h, False)
    clk = clocks.stop()
    step_infos = list(infos)
    x_check = xd[0].cpu().numpy() if rank == 0 else None  # first source's solution, for the oracle
    del bd, xd
    torch.cuda.empty_cache()

    # ---- end to end through the C ABI with pinned host buffers --------------------------
    bh = [torch.from_numpy(host_group(g)).pin_memory() for g in range(groups)]
    xh = torch.zeros(bh[0].shape, dtype=bh[0].dtype).pin_memory()
    step(bh[0], xh)
    sec_e2e = timed(args.steps, lambda i: step(bh[i % groups], xh))
    h2d = (bh[0].numel() + xh.numel()) * 16
    d2h = xh.numel() * 16
    del bh, xh
    scale = None
    if not args.no_scale_kernels:
        try:
            scale = kernels_on_workload(h, tm, wl, R, json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
                                        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {})
        except Exception as e:  # report, do not hide
            scale = {"error": str(e)[:300]}
    tm.tm_destroy(h)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    K = args.steps
    value = job_seconds_per_step(sec, world, K)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    outer_iters = sum(i["iters"] for i in step_infos) / K  # summed over the step's right-hand sides
    launches = sum(v["launches"] for v in prof.values())
    roof = None
    outer = {"iters": round(outer_iters / R), "restart": p.restart, "rhs": R, "steps": K}
    model = roofline_model(dom, dict(wl, block_oe=p.block_oe, sap1_prec=p.sap1_prec, mr_iters=p.mr_iters,
                                     outer_apply=p.outer_apply),
                           prof[dom]["units"], prof[dom]["launches"], outer, peaks)
    if model is not None and prof[dom]["launches"]:
        avg_s = prof[dom]["ms"] / prof[dom]["launches"] / 1000.0
        if dom == "coarse_oe":
            avg_s *= 2  # the model counts one Schur application (two launches)
        achieved = model["work"] / avg_s / 1e9
        tr = ncu_traffic(args.workload, dom)
        roof = {"kernel": dom, "bound": model["bound"], "achieved": round(achieved, 3), "peak": model["peak"],
                "unit": model["unit"], "frac": round(achieved / model["peak"], 4),
                "traffic": (tr * prof[dom]["units"] / prof[dom]["launches"]) if tr else None,
                ("flops_per_launch" if model["bound"] == "alu" else "bytes_per_launch"):
                    model["work"] * (1e3 if model["bound"] == "alu" else 1),
                "avg_launch_us": round(avg_s * 1e6, 2), "peak_source": model["peak_source"]}
        if "hbm_work" in model:  # the same launch against the HBM roof, in algorithmic bytes
            roof["hbm"] = {"bytes_per_launch": model["hbm_work"], "achieved_gbs": round(model["hbm_work"] / avg_s / 1e9, 1),
                           "frac": round(model["hbm_work"] / avg_s / 1e9 / model["hbm_peak"], 4)}
    tot_ms = sum(v["ms"] for v in prof_all.values())
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "share": round(v["ms"] / max(1e-12, tot_ms), 4)}
               for k, v in prof_all.items() if v["launches"]}
    counts = step_counts(prof, K, outer_iters, levels)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            costs = run_oracle_worker(args.workload)
            osec = oracle_seconds(costs, counts, wl)
            cpu = {"value": round(osec, 2), "unit": "s", "cores": 1, "kind": "oracle",
                   "sample": ("FP64 numpy oracle, one thread: per-site costs of each step component timed on "
                              "sample lattices (D apply, SAP colour, P, P^dagger, outer FGMRES iteration on "
                              "16^3x32" + ("; level-1 D_c1, level-1 SAP colour, P2, level-1 FGMRES iteration on "
                                           "8x4x4x4 level-1 sites; coarsest odd-even GMRES step on 4^4 sites"
                                           if levels == 3 else "; odd-even coarse GMRES steps")
                              + ") x the sites of this workload x this run's unit counts per step"),
                   "sample_wall_s": round(costs["_wall"], 1),
                   "unit_costs_s_per_site": {k: float(f"{v:.4g}") for k, v in costs.items() if not k.startswith("_")}}
        except Exception as e:  # report, do not hide
            cpu = {"value": None, "error": str(e)[:300]}
        if x_check is not None:
            try:
                b0 = host_group(0)[0]
                nw = min(16, os.cpu_count() or 1)
                rr, ts = oracle_true_residual(U, x_check.reshape(L + (4, 3)), b0.reshape(L + (4, 3)), m0,
                                              wl["c_sw"], wl["mu"], -1.0, nw)
                cpu = dict(cpu or {}, oracle_check={
                    "true_relres": rr, "seconds": round(ts, 1), "processes": nw,
                    "what": "the oracle's FP64 D(mu) recomputes ||b - D x|| / ||b|| of the first source's GPU "
                            "solution on the full lattice, T-slab by T-slab"})
            except Exception as e:  # report, do not hide
                cpu = dict(cpu or {}, oracle_check={"error": str(e)[:300]})
    if args.write_counts:
        os.makedirs(os.path.dirname(COUNTS_FILE), exist_ok=True)
        json.dump({"workload": args.workload, "counts_per_step": counts,
                   "note": "unit counts per step of the hot path on this workload (D applies, SAP colour "
                           "units, transfers, coarse steps, outer iterations), used to scale the oracle's "
                           "per-site costs"}, open(COUNTS_FILE, "w"), indent=1)
    setup_kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 1)} for k, v in prof_setup.items()
                     if v["launches"]}
    oa = "f32x2" if p.outer_apply == TM_F32X2 else "f64"
    line = {
        "metric": METRIC,
        "value": round(value, 5),
        "unit": "s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(sec / K * 1000, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": (f"f64 FGMRES vectors and true residual; {oa} D(mu) z_k products"
                  + (" and Arnoldi arithmetic" if oa == "f32x2" else "") + "; f32 K-cycle"
                  + (f"; {PREC_NAMES[p.sap_prec]} SAP links/clover/D_oo^-1" if p.sap_prec in (2, 3) else "")
                  + (f"; {PREC_NAMES[p.transfer_prec]} P for the transfers" if p.transfer_prec in (2, 3) else "")
                  + (f"; {PREC_NAMES[p.sap1_prec]} level-1 SAP blocks" if p.sap1_prec in (2, 3) else "")
                  + ("; tf32 coarsest Schur complement" if p.coarse_mma else "")),
        "data": f"synthetic (seeded random SU(3) field U = exp({wl['eps']} i H); "
                + ("12 spin-colour point sources)" if wl.get("point") else "Gaussian rhs)"),
        "config": {
            "workload": args.workload, "lattice_TZYX": list(L), "sites": V, "levels": levels,
            **({"nv2": wl["nv2"], "aggregate2": list(wl["agg2"]), "sap_block1": list(wl["sap_block1"]),
                "coarse_setup_iters": wl["coarse_setup_iters"],
                "sap1_prec": PREC_NAMES[p.sap1_prec]} if levels == 3 else {}),
            "sap_prec": PREC_NAMES[p.sap_prec], "transfer_prec": PREC_NAMES[p.transfer_prec],
            "nv": nv, "aggregate": list(wl["agg"]), "sap_block": list(wl["sap_block"]),
            "restart": p.restart, "coarse_tol": p.coarse_tol, "post_smooth": p.post_smooth, "mr_iters": p.mr_iters,
            "coarse_mma": p.coarse_mma, "outer_apply": oa, "block_oe": p.block_oe,
            "m0": m0, "m0_source": m0_src, "c_sw": wl["c_sw"], "mu": wl["mu"], "delta": wl["delta"],
            "setup_iters": wl["setup_iters"], "tol": wl["tol"], "rhs_total": nrhs, "rhs_per_step": R,
            "rhs": "12 spin-colour point sources" if wl.get("point") else "Gaussian",
            "step": (f"FGMRES solve of {R} right-hand side(s) to 1e-10 (one group of {nrhs}); gauge field, clover "
                     f"term and adaptive setup once before the timed steps (setup_s)"),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "every fine vector > 129 MB L2 (no extra flush)",
        },
        "setup_s": round(setup_s, 3),
        "setup_kernels": setup_kernels,
        "solve": {
            "outer_iters_per_step": [i["iters"] for i in step_infos],
            "coarse_iters_per_step": [i["coarse_iters"] for i in step_infos],
            "true_relres_max": max(i["true_relres"] for i in step_infos),
            "seconds_per_rhs": round(value / R, 4),
            "seconds_all_sources": round(value * nrhs / R, 3),
        },
        "e2e": {"value": round(job_seconds_per_step(sec_e2e, world, K), 5), "unit": "s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": f"steps cycle through the {groups} source group(s); x0 = 0 written on the host each step"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels_one_step": kernels,
        "kernels_on_workload": scale,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
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


def reference_config(name: str, wl: dict) -> dict:
    """The workload part of the native arm's config, from the workload table
    (the library's defaults where the table leaves a setting out)."""
    V, V1, V2 = volumes(wl)
    m0, m0_src = workload_m0(wl)
    nrhs = wl.get("nrhs", 1)
    cfg = {"workload": name, "lattice_TZYX": list(wl["L"]), "sites": V, "levels": wl.get("levels", 2),
           "nv": wl["nv"], "aggregate": list(wl["agg"]), "sap_block": list(wl["sap_block"]),
           "restart": wl.get("restart", 25), "coarse_tol": wl.get("coarse_tol", 0.05),
           "post_smooth": wl.get("post_smooth", 4), "mr_iters": 4, "block_oe": wl.get("block_oe", 0),
           "m0": m0, "m0_source": m0_src, "c_sw": wl["c_sw"], "mu": wl["mu"], "delta": wl["delta"],
           "setup_iters": wl["setup_iters"], "tol": wl["tol"], "rhs_total": nrhs,
           "rhs_per_step": wl.get("rhs_batch", nrhs),
           "rhs": "12 spin-colour point sources" if wl.get("point") else "Gaussian",
           "arithmetic": "FP64 numpy oracle (every step of the method in FP64)"}
    if cfg["levels"] == 3:
        cfg.update({"nv2": wl["nv2"], "aggregate2": list(wl["agg2"]), "sap_block1": list(wl["sap_block1"]),
                    "coarse_setup_iters": wl["coarse_setup_iters"]})
    return cfg


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if not os.path.exists(COUNTS_FILE):
        print(json.dumps({"impl": "reference", "unavailable":
                          "no unit counts recorded (profiles/bench_unit_counts.json)"}))
        return
    rec = json.load(open(COUNTS_FILE))
    if rec.get("workload") != args.workload:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"unit counts recorded for {rec.get('workload')}, not {args.workload}"}))
        return
    counts = rec["counts_per_step"]
    wl = WORKLOADS[args.workload]
    times = []
    last = None
    for i in range(args.warmup + args.steps):
        costs = run_oracle_worker(args.workload)
        if i >= args.warmup:
            times.append(oracle_seconds(costs, counts, wl))
        last = costs
    value = statistics.mean(times)
    print(json.dumps({
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 2), "unit": "s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": reference_config(args.workload, wl),
        "cpu_baseline": {"value": round(value, 2), "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": "per-site oracle costs on sample lattices x the workload's sites x the unit "
                                   "counts per step recorded from a GPU run (profiles/bench_unit_counts.json)",
                         "unit_costs_s_per_site": {k: float(f"{v:.4g}") for k, v in last.items()
                                                   if not k.startswith("_")}},
        "e2e": {"value": round(value, 2), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main_compare(args):
    """Fig. 1 shape (Sec. 1): time to solution of DD-alphaAMG, setup included,
    against oeCG for 1 and for all right-hand sides of the workload.  oeCG
    solves one right-hand side after another (FP32 CG inside FP64 defect
    correction); its time for n sources is n times the measured mean of the
    first sources.  One JSON line, not the bench line."""
    import numpy as np
    import torch
    import inputs
    import paper_1611_01034_gb300 as tm

    name = args.workload or "24x24x24x48_2lvl_nv24_12pt"
    wl = WORKLOADS[name]
    m0, m0_src = (args.m0, "command line") if args.m0 is not None else workload_m0(wl)
    L, nv, seed = wl["L"], wl["nv"], wl["seed"]
    U = inputs.gauge_field(L, wl["eps"], seed, workers=min(16, os.cpu_count() or 1))
    torch.cuda.set_device(0)
    levels = wl.get("levels", 2)
    nrhs = wl.get("nrhs", 1)
    R = args.rhs_batch or wl.get("rhs_batch", nrhs)
    V, V1, V2 = volumes(wl)
    n_w = wl["nv2"] * V1 * 2 * nv if levels == 3 else 0
    tv_host = None
    if not wl.get("device_inputs"):
        tv_host = inputs.random_test_vectors(L, nv, seed + inputs.TV_SEED_OFFSET)
        if levels == 3:
            Lc1 = tuple(L[d] // wl["agg"][d] for d in range(4))
            w0 = inputs.random_coarse_vectors(Lc1, 2 * nv, wl["nv2"], seed + inputs.TV_SEED_OFFSET + 1)
            tv_host = np.concatenate([tv_host.ravel(), w0.ravel()])

    def make_tv():  # as in the benchmark: the 48^3 x 96 test vectors are drawn on the device
        if tv_host is not None:
            return torch.from_numpy(tv_host).cuda()
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed + inputs.TV_SEED_OFFSET)
        return torch.randn((nv * V * 12 + n_w,), dtype=torch.complex128, device="cuda", generator=gen)

    x0 = inputs.point_source_site(L, seed + inputs.RHS_SEED_OFFSET) if wl.get("point") else None

    def sources(first, n):
        if x0 is not None:
            return point_source_group(L, x0, first, n)
        return inputs.gaussian_spinor(L, seed + inputs.RHS_SEED_OFFSET + first, nrhs=n).reshape(n, V, 4, 3)

    stream = torch.cuda.current_stream()
    extra = {k: wl[k] for k in ("nv2", "agg2", "sap_block1", "coarse_setup_iters", "restart", "sap1_prec",
                                "outer_apply", "block_oe", "sap_prec", "transfer_prec", "coarsest_steps", "post_smooth",
                                "coarse_tol") if k in wl}
    extra["coarse_mma"] = wl.get("coarse_mma", 0)
    for kv in args.param or []:
        k, v = kv.split("=", 1)
        extra[k] = float(v) if "." in v or "e" in v else int(v)
    extra.setdefault("cycle_prec", tm.TM_F32)
    p = tm.params(L=L, m0=m0, c_sw=wl["c_sw"], mu=wl["mu"], delta=wl["delta"], nv=nv, agg=wl["agg"],
                  sap_block=wl["sap_block"], setup_iters=wl["setup_iters"], max_rhs=R, levels=levels, **extra)
    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    def new_setup():  # a handle with the gauge field and the adaptive setup; returns (handle, seconds)
        hh = tm.tm_create(p, stream)
        tvd = make_tv()
        Ud = torch.from_numpy(U).cuda()  # only while the setup runs: the 48^3 x 96 solves need the room
        t, _ = timed(lambda: (tm.tm_load_gauge(hh, Ud), tm.tm_setup(hh, tvd)))
        del tvd, Ud
        torch.cuda.empty_cache()
        return hh, t

    # DD-alphaAMG, all sources R at a time (the handle's batch), inputs resident on the device
    h, t_setup_a = new_setup()
    t_amgn, it_n, res_n = 0.0, 0, 0.0
    for g0 in range(0, nrhs, R):
        n = min(R, nrhs - g0)
        bg = torch.from_numpy(sources(g0, n)).cuda()
        xg = torch.zeros_like(bg)
        t, (st, info) = timed(lambda: tm.tm_solve(h, bg, xg, n, wl["tol"]))
        if st != tm.TM_OK:
            raise RuntimeError(tm.tm_last_error(h))
        t_amgn += t
        it_n += info.iters
        res_n = max(res_n, info.true_relres)
        del bg, xg
    tm.tm_destroy(h)
    torch.cuda.empty_cache()
    # DD-alphaAMG, one source, on a fresh handle (its single-rhs work buffers would not fit next to the batch's)
    h, t_setup = new_setup()
    b1 = torch.from_numpy(sources(0, 1)).cuda()
    x1 = torch.zeros_like(b1)
    t_amg1, (st, info1) = timed(lambda: tm.tm_solve(h, b1, x1, 1, wl["tol"]))
    if st != tm.TM_OK:
        raise RuntimeError(tm.tm_last_error(h))
    del b1, x1
    tm.tm_destroy(h)
    torch.cuda.empty_cache()
    # oeCG needs only the gauge field: a handle without a hierarchy worth the name
    pc = tm.params(L=L, m0=m0, c_sw=wl["c_sw"], mu=wl["mu"], delta=1.0, nv=1, agg=wl["agg"],
                   sap_block=wl["sap_block"], max_rhs=1, cycle_prec=tm.TM_F32)
    h = tm.tm_create(pc, stream)
    tm.tm_load_gauge(h, torch.from_numpy(U).cuda())
    torch.cuda.empty_cache()
    n_cg = min(2, nrhs)
    t_cg = []
    cg_iters = []
    cg_res = 0.0
    for r in range(n_cg):
        br = torch.from_numpy(sources(r, 1)).cuda()
        xr = torch.zeros_like(br)
        t, (st, info) = timed(lambda: tm.tm_solve_oecg(h, br, xr, 1, wl["tol"]))
        if st != tm.TM_OK:
            raise RuntimeError(tm.tm_last_error(h))
        t_cg.append(t)
        cg_iters.append(info.iters)
        cg_res = max(cg_res, info.true_relres)
    cg_per_rhs = statistics.mean(t_cg)
    rows = []
    for n, t_solve in ((1, t_amg1), (nrhs, t_amgn)):
        amg = t_setup + t_solve
        rows.append({"nrhs": n, "amg_s": round(amg, 4), "oecg_s": round(n * cg_per_rhs, 4),
                     "speedup": round(n * cg_per_rhs / amg, 2)})
    print(json.dumps({
        "metric": "time to solution to 1e-10: DD-alphaAMG (setup included) vs oeCG, Fig. 1 shape",
        "unit": "s", "workload": name, "m0": m0, "m0_source": m0_src, "mu": wl["mu"],
        "amg_setup_s": round(t_setup, 4), "amg_setup_first_s": round(t_setup_a, 4),
        "amg_solve_1_s": round(t_amg1, 4),
        "amg_solve_all_s": round(t_amgn, 4), "rhs_all": nrhs,
        "amg_outer_iters_per_rhs": round(it_n / nrhs, 2),
        "oecg_s_per_rhs": [round(t, 4) for t in t_cg], "oecg_cg_iters_per_rhs": cg_iters,
        "true_relres": {"amg": res_n, "oecg": cg_res},
        "rows": rows,
        "timing": "wall clock around each call with a device synchronisation on both sides",
    }), flush=True)
    tm.tm_destroy(h)


def main_check_m0(args):
    """Check of the near-critical m0 on the workload's own lattice: inverse
    iteration with the library's squared solve, y = (D(mu)^dagger D(mu))^-1 x,
    which shares its low modes with D_W^dagger D_W (D^dagger D = D_W^dagger D_W
    + mu^2).  After k steps 1 / |y| (x normalised) bounds the lowest eigenvalue
    lambda of D^dagger D from above, hence sigma_min(D_W) <= sqrt(1/|y| - mu^2).
    One JSON line, not the bench line."""
    import numpy as np
    import torch
    import inputs
    import paper_1611_01034_gb300 as tm

    name = args.workload or DEFAULT_WORKLOAD
    wl = WORKLOADS[name]
    m0, m0_src = (args.m0, "command line") if args.m0 is not None else workload_m0(wl)
    L, nv, seed = wl["L"], wl["nv"], wl["seed"]
    U = inputs.gauge_field(L, wl["eps"], seed, workers=min(16, os.cpu_count() or 1))
    torch.cuda.set_device(0)
    levels = wl.get("levels", 2)
    V, V1, V2 = volumes(wl)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + inputs.TV_SEED_OFFSET)
    n_w = wl["nv2"] * V1 * 2 * nv if levels == 3 else 0
    tvd = torch.randn((nv * V * 12 + n_w,), dtype=torch.complex128, device="cuda", generator=gen)
    extra = {k: wl[k] for k in ("nv2", "agg2", "sap_block1", "coarse_setup_iters", "restart", "sap1_prec",
                                "outer_apply", "block_oe", "sap_prec", "transfer_prec", "coarsest_steps", "post_smooth",
                                "coarse_tol") if k in wl}
    extra["coarse_mma"] = wl.get("coarse_mma", 0)
    extra.setdefault("cycle_prec", tm.TM_F32)
    p = tm.params(L=L, m0=m0, c_sw=wl["c_sw"], mu=wl["mu"], delta=wl["delta"], nv=nv, agg=wl["agg"],
                  sap_block=wl["sap_block"], setup_iters=wl["setup_iters"], max_rhs=1, levels=levels, **extra)
    stream = torch.cuda.current_stream()
    h = tm.tm_create(p, stream)
    tm.tm_load_gauge(h, torch.from_numpy(U).cuda())
    tm.tm_setup(h, tvd)
    del tvd
    torch.cuda.empty_cache()
    gen.manual_seed(seed + 7777)
    x = torch.randn((1, V, 4, 3), dtype=torch.complex128, device="cuda", generator=gen)
    x /= torch.linalg.vector_norm(x)
    mu = wl["mu"]
    rows = []
    t0 = time.time()
    for k in range(1, args.m0_iters + 1):
        y = torch.zeros_like(x)
        st, info = tm.tm_solve_squared(h, x, y, 1, 1e-8)
        if st != tm.TM_OK:
            raise RuntimeError(tm.tm_last_error(h))
        ny = float(torch.linalg.vector_norm(y))
        rq = float(torch.vdot(x.flatten(), y.flatten()).real)
        lam = 1.0 / ny
        rows.append({"k": k, "lambda_upper": lam, "sigma_w_upper": float(np.sqrt(max(lam - mu * mu, 0.0))),
                     "rayleigh_inverse": rq, "outer_iters": info.iters})
        x = y / ny
    print(json.dumps({
        "metric": "upper bound of sigma_min(D_W(m0)) by inverse iteration on D(mu)^dagger D(mu)",
        "workload": name, "m0": m0, "m0_source": m0_src, "mu": mu, "target_sigma_min": 1e-3,
        "iterations": rows, "seconds": round(time.time() - t0, 1),
        "reading": "D^dagger D = D_W^dagger D_W + mu^2, so lambda_min(D^dagger D) <= 1/|y_k| gives "
                   "sigma_min(D_W) <= sqrt(1/|y_k| - mu^2); the bound falls towards sigma_min as k grows"}),
          flush=True)
    tm.tm_destroy(h)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=None, choices=list(WORKLOADS),
                    help="default: the 48^3 x 96 three-level workload (24^3 x 48 with --compare-oecg)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--write-counts", action="store_true")
    ap.add_argument("--param", action="append", help="override a tm_params field: name=value")
    ap.add_argument("--rhs-batch", type=int, default=None, help="right-hand sides per step")
    ap.add_argument("--no-scale-kernels", action="store_true",
                    help="skip the D(mu) and D_c1 measurements on the workload's lattice")
    ap.add_argument("--oracle-worker", default=None)
    ap.add_argument("--m0", type=float, default=None, help="override the workload's tuned m0")
    ap.add_argument("--compare-oecg", action="store_true",
                    help="Fig. 1 shape: DD-alphaAMG (with setup) against oeCG on --workload (default 24^3 x 48)")
    ap.add_argument("--check-m0", action="store_true",
                    help="inverse iteration on D(mu)^dagger D(mu): an upper bound of sigma_min(D_W(m0))")
    ap.add_argument("--m0-iters", type=int, default=6)
    ap.add_argument("--coarse-mma", type=int, default=None,
                    help="override the workload's coarse_mma (0 CUDA cores, 1..3 TF32 tensor-core products)")
    args = ap.parse_args()
    if args.oracle_worker:
        print(json.dumps(oracle_unit_costs(args.oracle_worker)))
        return
    if args.compare_oecg:
        main_compare(args)
        return
    if args.check_m0:
        main_check_m0(args)
        return
    args.workload = args.workload or DEFAULT_WORKLOAD
    if args.impl == "reference":
        main_reference(args)
    elif args.workload == "16x16x16x16_learned":
        main_learned(args)
    else:
        main_native(args)


if __name__ == "__main__":
    main()
