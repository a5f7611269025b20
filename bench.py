#!/usr/bin/env python
"""Benchmark: GW iterations/s on the five-orbital 32x32x8 DLR workload.

One step = one full GW iteration through qa_gw_step (G -> P -> W -> Sigma ->
Dyson -> mu -> G) on the mixed-precision path, inputs resident in HBM; the
steps alternate between two fixed inputs, G0 and its first iteration.  The
headline is the accurate mixed path (QA_MIXED: double-float storage and
FP32-based arithmetic, tensor-core DLR maps from fixed-point bf16 slices, the
Dyson-W solve in FP32 refined by a double-float residual step), which holds
Sigma within 1e-7 of the FP64 oracle; its measured error against the oracle on
a small workload is part of the line.  The library's default pair basis for it
is the exact reduced one (rho = 15 of the 25 pairs, W^C = B Wt^C B^H; see
include/qa.h, qa_set_pair_basis).  The same line reports, beside the headline,
the FP32 fast mode (QA_FP32, complex64, ~1e-6 - 1e-5 of FP64) and the FP64 path
on both bases.  It also carries the end-to-end number through the public API
with host buffers, the per-stage times, the roofline of the dominant kernel
against FMA rates measured in the same run, sampled clocks and the CPU oracle
baseline (complete iterations on two smaller workloads, one thread and all
cores, plus a sampled model of the 32x32x8 iteration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank runs an independent replica of
the workload (the iteration has no cross-GPU exchange at this size); value is
the total iterations of all ranks divided by the slowest rank's time.
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
sys.path.insert(0, ROOT)

METRIC = "GW iterations/s (5-orbital, 32×32×8 k, DLR) mixed vs FP64; % of HBM roofline"
UNIT = "GW iterations/s"
WORKLOAD = "five-orbital-32x32x8"


# ------------------------------------------------------------------ helpers

def peaks(measure_alu=True):
    """HBM and bf16 peaks from MEASURED_PEAKS.json (driver-written; fallback
    6.8 TB/s and 1.9 PFLOP/s), FP32 and FP64 FMA rates measured in this run with
    qa_fma_probe (eight independent FMA chains per thread, 8 blocks per SM)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        pk = {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d.get("bf16_tflops_sustained", d.get("bf16_tflops")),
              "src": "measured"}
    else:
        pk = {"hbm_gbs": 6800.0, "bf16_tflops": 1700.0, "src": "fallback"}
    if measure_alu:
        from paper_2604_22223_gb300 import qa
        pk["fp32_tflops"], pk["fp32_probe_ms"] = qa.fma_rate("fp32", iters=8192)
        pk["fp64_tflops"], pk["fp64_probe_ms"] = qa.fma_rate("fp64", iters=256)
        pk["alu_src"] = "measured in this run (qa_fma_probe FMA chains, best of 3)"
    return pk


CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def summarise_clock_rows(rows, t0, t1):
    """Median SM clock, max clock and active throttle reasons of the nvidia-smi
    rows (timestamp, index, clocks.sm, clocks.max.sm, power, active, the four
    reasons) sampled inside the host window [t0, t1]; when no sample falls
    inside, the one closest to the window's middle stands in for it."""
    import datetime
    parsed = []
    for r in rows:
        if len(r) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            sm, mx = float(r[2]), float(r[3])
        except ValueError:
            continue
        parsed.append((ts, sm, mx, [v.strip().lower() == "active" for v in r[6:10]]))
    inside = [p for p in parsed if t0 <= p[0] <= t1]
    if not inside and parsed:
        mid = 0.5 * (t0 + t1)
        inside = [min(parsed, key=lambda p: abs(p[0] - mid))]
    reasons = sorted({nm for p in inside for nm, on in zip(CLOCK_REASONS, p[3]) if on})
    return {"sm_mhz": statistics.median(p[1] for p in inside) if inside else None,
            "sm_max_mhz": max(p[2] for p in inside) if inside else None, "reasons": reasons,
            "samples": len(inside), "window_s": round(t1 - t0, 3)}


class Clocks:
    """nvidia-smi sampling (every 100 ms) around the timed region: started before
    the warm-up, its samples are kept when their timestamps fall inside the
    host-clock window that brackets the timed steps."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001 - clocks are best effort
            self.proc = None
            return
        # wait (at most 5 s) until the sampler writes its first row
        for _ in range(100):
            if self.proc.poll() is not None or os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.05)

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)                     # one more sample after the window
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        t0 = self.t0 if self.t0 is not None else 0.0
        t1 = self.t1 if self.t1 is not None else time.time()
        return summarise_clock_rows(rows, t0, t1)


def s_block_sizes(ctx):
    """Size of the diagonal block of S = B^H V(R) B (all listed R) containing each
    reduced index: indices coupled by a non-zero entry, connected components."""
    import numpy as np
    B = ctx.basis
    rho = B.shape[1]
    parent = list(range(rho))

    def root(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for V in np.asarray(ctx.model.V):
        S = B.conj().T @ V @ B
        for i, k in zip(*np.nonzero(np.abs(S) > 0)):
            parent[root(int(i))] = root(int(k))
    roots = [root(i) for i in range(rho)]
    return [roots.count(roots[i]) for i in range(rho)]


def s_is_real(ctx):
    """S(q) = B^H V(q) B is real when every S(R) is real with S(-R) = S(R) (the
    test the library applies to take its real-S Dyson-W variant)."""
    import numpy as np
    m = ctx.model
    B = ctx.basis if ctx.reduced else np.eye(ctx.npair)
    S = [B.conj().T @ V @ B for V in np.asarray(m.V)]
    idx = {tuple(R): i for i, R in enumerate(np.asarray(m.V_R))}
    for i, R in enumerate(np.asarray(m.V_R)):
        j = idx.get(tuple(-R))
        if j is None or np.any(S[i].imag != 0) or np.any(S[i] != S[j]):
            return False
    return len(S) > 0


def stage_costs(ctx, prec):
    """Algorithmic bytes and arithmetic per launch of each big-tensor stage.

    X = r nb^2 N_k big-tensor elements (nb = rho on the reduced basis, npair on
    the full one), Y = r norb^2 N_k small-tensor elements; es = 16 B (FP64 and
    the double-float mixed path) or 8 B (FP32).  Arithmetic is a pair (count,
    kind): "fp64" / "fp32" floating-point operations; "df" FP32 instructions of
    the double-float algorithm (one each; a TwoSum is 6, a TwoProd 2, a complex
    multiply-add of a double-float by an FP32 value 40 and of two double-floats
    48, a complex double-float add 22, a complex double-float product 38);
    "tensor" bf16 tensor-core flops.  On grids of power-of-two axes the bubble
    is produced inside the R -> q FFT (one launch, reported under fft_R_to_q)."""
    import math
    r, nk, no, nb = ctx.r, ctx.nk, ctx.norb, ctx.nb
    es = 8 if prec == "fp32" else 16
    X = r * nb * nb * nk
    Y = r * no * no * nk
    lg = math.log2(nk)
    n = nb
    blk = s_block_sizes(ctx) if ctx.reduced else [n] * n
    sb = sum(blk)                                   # non-zeros of S (per row: its block width)
    nterm = no ** 4                                 # Sigma terms per (R, tau)
    if prec == "mixed":
        # Dyson-W: FP32 formation (S P, S P S over the blocks of S), Gauss-Jordan on
        # [A | B] and the replay on R (FP32 complex multiply-adds, 4 instructions);
        # the residual R = M Y - X0: M = S P in double-float (48 per complex
        # multiply-add over the non-zeros of S), Y = S + X0, five bf16 slices of
        # both (4 instructions per slice and real value, one pack per two) and the
        # double-float sum of the five level results (4 TwoSums and a renormalisation
        # per real output, 30); the slice products themselves run on the tensor
        # cores (15 slice pairs x 4 real 16x16x16 products per system, not counted here)
        # (with a real S(q), M = S P takes two real products per entry instead of four)
        f32c = 2 * n * sb + sum((n - 1) * ((n - 1 - c) + n) for c in range(n)) + n * (n - 1) * n
        mform = 24 if (ctx.reduced and n == 15 and s_is_real(ctx)) else 48
        dyson = (r * nk * (4 * f32c + mform * n * sb + 2 * (2 * n * n) * (5 * 4 + 3) + 2 * n * n * 30
                           + 10 * n * n), "df")
        kp = (2 * r + 15) // 16 * 16
        dlr = (15 * 2 * (nb * nb * nk) * kp * kp, "tensor")      # 15 slice products, M x N x K
        fft = (60 * X * lg, "df")                                # ~60 per point and radix-2 stage
        sig = (86 * nterm * r * nk, "df")
        bub = (100 * X, "df")
    else:
        fd = 8 * (n ** 3 + (n ** 3 if prec == "fp32" else 0) + n ** 3 / 3 + n ** 3)   # VP, [VPV], LU, solve
        if prec == "fp32" and ctx.reduced and n <= 16:
            # the FP32 tile kernel: S P and S P S over the diagonal blocks of S only, then
            # Gauss-Jordan on [A | B] (n - 1 rows x (2n - 1 - c) entries per column c) and
            # the final row scaling
            fd = 8 * (2 * n * sb + (n - 1) * n * (3 * n - 1) / 2 + n * n)
        dyson = (r * nk * fd, prec)
        dlr = (8 * r * X, prec)
        fft = (5 * X * lg, prec)
        sig = (8 * nterm * r * nk, prec)
        bub = (6 * X, prec)
    return {
        "bubble": (X * es + 2 * Y * es, bub),
        "fft_R_to_q": (X * es + 2 * Y * es, (fft[0] + bub[0], fft[1])),
        "dlr_tau_to_nu": (2 * X * es, dlr),
        "dyson_w": (2 * X * es + nk * n * n * es, dyson),
        "dlr_nu_to_tau": (2 * X * es, dlr),
        "fft_q_to_R": (2 * X * es, fft),
        "sigma": (X * es + 2 * Y * es, sig),
    }


def iteration_bytes(ctx, prec):
    """Minimum HBM bytes of one iteration: P and W^C written and read once each
    (in the basis and precision the path stores), about six passes over the
    small G/Sigma tensors (complex128) and V(q)."""
    r, nk, no, nb = ctx.r, ctx.nk, ctx.norb, ctx.nb
    X = r * nb * nb * nk
    Y = r * no * no * nk
    return 4 * X * (8 if prec == "fp32" else 16) + 6 * Y * 16 + nk * nb * nb * 16


def roofline(ctx, prec, stage_ms, pk):
    costs = stage_costs(ctx, prec)
    name = max(costs, key=lambda s: stage_ms.get(s, 0.0))
    ms = stage_ms[name]
    b, (f, kind) = costs[name]
    peak = {"fp64": pk["fp64_tflops"], "fp32": pk["fp32_tflops"], "df": pk["fp32_tflops"] / 2,
            "tensor": pk["bf16_tflops"]}[kind]
    t_hbm = b / (pk["hbm_gbs"] * 1e9)
    t_alu = f / (peak * 1e12)
    if t_hbm >= t_alu:
        out = {"bound": "hbm", "achieved": b / (ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
               "peak_src": pk["src"] + " hbm_gbs (MEASURED_PEAKS.json)"}
    else:
        out = {"bound": "tensor" if kind == "tensor" else "alu", "achieved": f / (ms * 1e-3) / 1e12,
               "peak": peak, "unit": "TFLOP/s",
               "peak_src": {"fp64": "FP64 FMA rate " + pk["alu_src"],
                            "fp32": "FP32 FMA rate " + pk["alu_src"],
                            "df": "FP32 FMA instruction rate (half the FP32 flop rate) " + pk["alu_src"],
                            "tensor": pk["src"] + " bf16 sustained (MEASURED_PEAKS.json)"}[kind]}
        if kind == "df":
            out["work"] = "FP32 instructions of the double-float algorithm, counted one op each"
    out["frac"] = out["achieved"] / out["peak"]
    out["kernel"] = name
    out["ms_per_launch"] = ms
    out["algorithmic_bytes"] = b
    out["algorithmic_ops"] = f
    out["ops_kind"] = kind
    out["traffic"] = traffic_for(name, prec)
    return out


def traffic_for(stage, prec):
    """DRAM bytes per launch of a stage's kernel at the bench workload, from a
    committed ncu summary (entries keyed "<precision>:<stage>"); None when the
    kernel's sources changed since (the summary records a SHA-256 of their
    contents)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        ent = json.load(open(p)).get("%s:%s" % (prec, stage))
        if not ent:
            return None
        h = hashlib.sha256()
        for rel in ent["sources"]:
            with open(os.path.join(ROOT, rel), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != ent["source_sha256"]:
            return None
        return ent["dram_bytes_per_launch"]
    except Exception:  # noqa: BLE001
        return None


def oracle_sample(model, n_q=1, n_k=1):
    """Time the CPU oracle on a bounded sample of the workload and extrapolate.

    Per iteration the explicit-sum oracle does, for every q, the bubble k-sum,
    the DLR transform and the W Dyson solve (polarization_at_q +
    screened_interaction), for every k the Sigma q-sum (self_energy_at_k), and
    ~45 density evaluations of the mu bisection.  Stand-in arrays of the
    workload's shapes are used (cost does not depend on values)."""
    import numpy as np
    from oracle import gw, lattice
    dlr = gw.make_dlr(model)
    rng = np.random.default_rng(0)
    nk, r, no, npair = model.nk, dlr.r, model.norb, model.npair
    G = rng.normal(size=(nk, r, no, no)) + 1j * rng.normal(size=(nk, r, no, no))
    t0 = time.perf_counter()
    Grefl = gw.reflected(model, dlr, G)
    t_shared = time.perf_counter() - t0
    Vq = lattice.V_q(model)
    tq = []
    for iq in range(n_q):
        t0 = time.perf_counter()
        P = gw.polarization_at_q(model, dlr, G, iq, Grefl)
        gw.screened_interaction(Vq[iq:iq + 1], P[None])
        tq.append(time.perf_counter() - t0)
    WC = np.zeros((nk, r, npair, npair), dtype=np.complex128)
    tk = []
    for ik in range(n_k):
        t0 = time.perf_counter()
        gw.self_energy_at_k(model, G, WC, ik)
        tk.append(time.perf_counter() - t0)
    del WC
    Hk = lattice.H_k(model)
    t0 = time.perf_counter()
    gw.density_from_iw(dlr, gw.g_iw(dlr, Hk, 0.0))
    t_dens = time.perf_counter() - t0
    n_bis = 45
    t_iter = t_shared + nk * (statistics.mean(tq) + statistics.mean(tk)) + n_bis * t_dens
    return t_iter, {"t_q_s": statistics.mean(tq), "t_k_s": statistics.mean(tk),
                    "t_density_s": t_dens, "t_shared_s": t_shared}


# --------------------------------------------------------------- the arms

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(pg, value, device=None):
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def _event_ms(fn, reps=1):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    out = None
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def hf_qp_timing(ctx, pk):
    """The Hartree-Fock loop (qa_hf_solve, from the Fermi-Dirac density of H0
    to max |dSigma^HF| <= 1e-10, plain iteration) and the quasiparticle
    quantities (qa_qp) of the last GW step, on the bench workload.  The QP
    node sums read Sigma^C(k, i w) once: r norb^2 N_k elements."""
    from paper_2604_22223_gb300 import qa
    ctx.step()                                   # a fresh Sigma^C for qa_qp
    ctx.qp()                                     # warm-up
    ms_qp, _ = _event_ms(ctx.qp, reps=5)
    es = 8 if ctx.precision == qa.QA_FP32 else 16
    no2 = ctx.norb * ctx.norb
    qp_bytes = ctx.r * no2 * ctx.nk * es + 2 * no2 * ctx.nk * 16 * 2 + 5 * ctx.nk * no2 * 16
    ctx.hf_solve(500, 1e-10, 1.0, check=False)  # warm-up
    ms_hf, res = _event_ms(lambda: ctx.hf_solve(500, 1e-10, 1.0, check=False))
    _, mu, _, iters, resid, status = res
    return {"hf_ms": ms_hf, "hf_iterations": iters, "hf_ms_per_iteration": ms_hf / max(iters, 1),
            "hf_resid": resid, "hf_status": status, "hf_mu": mu,
            "qp_ms": ms_qp, "qp_algorithmic_bytes": qp_bytes,
            "qp_hbm_frac": qp_bytes / (ms_qp * 1e-3) / 1e9 / pk["hbm_gbs"],
            "note": "HF: per iteration one eigendecomposition of H0 + Sigma^HF per k (FP64 Jacobi), "
                    "a host-driven mu search over device Fermi-Dirac sums, n(k), Sigma^H/Sigma^F; "
                    "QP: node sums + per-k Z, Sigma(0), H_QP, eps; times are whole API calls"}


def paper_table1(qa, wl, dev, pg, world, timed):
    """One GW iteration on the paper's own benchmark model (degenerate
    five-orbital Hund-Hubbard, 8x8x8 k, beta = 100/eV, Lambda = 25 eV), both
    precisions; the paper's DLR+Vec time (Table 1, hardware not stated) is
    context, not a baseline."""
    import torch
    m = wl.config("five-orbital-paper-8x8x8")
    out = {"workload": "five-orbital-paper-8x8x8", "paper_dlr_vec_seconds_per_iteration": 232.56}
    for prec in ("mixed", "fp32", "fp64"):
        c = qa.Context(m, prec, device=str(dev))
        K = 10
        ms, stg, _, _, _ = timed(c, K, 3)
        ms = max_over_ranks(pg, ms, dev)
        out[prec] = {"ms_per_iteration": ms / K, "iterations_per_s": world * K / (ms / 1e3),
                     "dlr_rank": c.r, "pair_basis": "reduced rho=%d" % c.rho if c.reduced else
                     "full npair=%d" % c.npair}
        del c
        torch.cuda.empty_cache()
    return out


def barrier(pg):
    if pg is not None:
        pg.barrier()


def accuracy_check(qa, wl, dev):
    """Errors of the mixed and FP32 paths against the FP64 oracle (relative
    max-norm, one iteration from G0) on a small workload the oracle finishes in
    about a second: the accuracy the headline's speed comes with."""
    import numpy as np
    import torch
    from oracle import gw
    name = "five-orbital-4x3x2"
    m = wl.config(name)
    d = gw.make_dlr(m)
    G0, _ = gw.g0(m, d)
    o = gw.gw_step(m, d, G0)
    kl = lambda x: np.moveaxis(x, 0, -1)
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    out = {"workload": name, "reference": "FP64 CPU oracle (oracle/gw.py)"}
    for prec in ("mixed", "fp32"):
        c = qa.Context(m, prec, device=str(dev))
        G, mu, _, _ = c.step()
        W = c.get(qa.QA_WC_RTAU).cpu().numpy()
        if c.reduced:
            W = np.einsum("ai,...ijk,bj->...abk", c.basis, W, c.basis.conj())
        out[prec] = {"sigc_ktau": rel(c.get(qa.QA_SIGC_KTAU).cpu().numpy(), kl(o["sigc_ktau"])),
                     "sigc_kiw": rel(c.get(qa.QA_SIGC_KIW).cpu().numpy(), kl(o["sigc_kiw"])),
                     "WC_Rtau": rel(W, kl(o["WC_Rtau"])),
                     "G": rel(G.cpu().numpy(), kl(o["G_ktau"])),
                     "mu": abs(mu - o["mu"]) / max(1.0, abs(o["mu"]))}
        del c
        torch.cuda.empty_cache()
    out["stated_bound_sigma_mixed"] = 1e-7
    return out


def cpu_complete(name, threads):
    """Wall seconds of one complete oracle iteration (gw_step from G0) in a
    fresh interpreter; threads = 1 pins OpenMP/BLAS to one thread, None keeps
    the libraries' defaults (numpy's BLAS and LAPACK calls on all cores)."""
    env = dict(os.environ)
    if threads:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    code = ("import sys, time; sys.path.insert(0, %r); import workloads as wl; from oracle import gw; "
            "m = wl.config(%r); d = gw.make_dlr(m); G0, _ = gw.g0(m, d); t0 = time.perf_counter(); "
            "gw.gw_step(m, d, G0); print(time.perf_counter() - t0)") % (ROOT, name)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    return float(p.stdout.strip().splitlines()[-1])


def cpu_baseline_block(qa, wl, dev, timed_gpu):
    """Complete oracle iterations on two smaller workloads (one thread and all
    cores), the GPU's time on the same workloads, and the sampled model of the
    32x32x8 iteration (checked against the measured 16x16 iteration)."""
    model = wl.config(WORKLOAD)
    t_iter, parts = oracle_sample(model)
    complete = {}
    for name in ("square-8x8", "five-orbital-16x16"):
        one = cpu_complete(name, 1)
        allc = cpu_complete(name, None)
        m = wl.config(name)
        model_s, _ = oracle_sample(m)
        gpu_ms = timed_gpu(m)
        complete[name] = {"seconds_1_thread": one, "seconds_all_cores": allc,
                          "gpu_mixed_ms": gpu_ms, "sampled_model_seconds": model_s,
                          "model_over_measured_1_thread": model_s / one}
    return {"value": 1.0 / t_iter, "unit": UNIT,
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": "value: the FP64 explicit-sum oracle's 32x32x8 iteration modelled from timed "
                      "samples (bubble + DLR + W Dyson of 1 q-point, Sigma q-sum of 1 k-point, 1 density "
                      "evaluation), extrapolated to 8192 q, 8192 k and 45 bisection steps (numpy default "
                      "threading); complete_iterations: measured gw_step wall times (one thread: "
                      "OMP/OPENBLAS/MKL_NUM_THREADS=1; all cores: library defaults)",
            "modelled_seconds_per_iteration": t_iter, "model_parts": parts,
            "complete_iterations": complete}


def run_ours(args):
    import torch
    import workloads as wl
    from paper_2604_22223_gb300 import build, qa
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build()
    model = wl.config(WORKLOAD)
    pk = peaks()

    def timed(ctx, K, W, clocks=None):
        """W untimed + K timed iterations.  Step i takes input G_a (= G0) or
        G_b (= the iteration of G0) alternately, so every step is one full
        iteration over a fixed synthetic input and the mu search starts from
        the other input's chemical potential."""
        Ga = ctx.get(qa.QA_G0).clone()
        Gb = ctx.new_g()
        Gout = ctx.new_g()
        if clocks:
            clocks.start()                   # sampling before the warm-up
        ctx.step(Ga, Gb)
        for i in range(max(W - 1, 0)):
            ctx.step(Ga if i % 2 else Gb, Gout)
        stage = {}
        launches = 0
        evals = []
        barrier(pg)
        torch.cuda.synchronize()
        if clocks:
            clocks.begin()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(K):
            _, mu, n, st = ctx.step(Ga if i % 2 else Gb, Gout, timing=True)
            for k, v in st["stage_ms"].items():
                stage[k] = stage.get(k, 0.0) + v
            launches += st["launches"]
            evals.append(st["mu_evals"])
        e1.record()
        torch.cuda.synchronize()
        if clocks:
            clocks.end()
        ck = clocks.stop() if clocks else None
        barrier(pg)
        ms = e0.elapsed_time(e1)
        return ms, {k: v / K for k, v in stage.items()}, launches, evals, ck

    # the accurate mixed path on the default (reduced) pair basis: the headline
    ctx = qa.Context(model, "mixed", device=str(dev))
    clocks = Clocks(local)
    ms_mixed, stage_mixed, launches, evals, ck = timed(ctx, args.steps, args.warmup, clocks)
    ms_mixed = max_over_ranks(pg, ms_mixed, dev)
    value = world * args.steps / (ms_mixed / 1e3)
    rl = roofline(ctx, "mixed", stage_mixed, pk)
    it_bytes = iteration_bytes(ctx, "mixed")
    # end to end through the public API with pinned host buffers: every step copies its
    # input G host -> device and its output G device -> host.  Serial: copy, step, copy on
    # one stream.  Pipelined: the copies run on a second stream, the input of step i + 1
    # and the output of step i - 1 moving while step i computes (double-buffered).
    Gh_in = ctx.get(qa.QA_G0).cpu().pin_memory()
    Gh_out = [torch.empty_like(Gh_in).pin_memory() for _ in range(2)]
    Gd_in, Gd_out = [ctx.new_g(), ctx.new_g()], [ctx.new_g(), ctx.new_g()]
    for _ in range(2):
        Gd_in[0].copy_(Gh_in, non_blocking=True)
        ctx.step(Gd_in[0], Gd_out[0])
        Gh_out[0].copy_(Gd_out[0], non_blocking=True)
    torch.cuda.synchronize()
    K2 = max(2, args.steps // 2)
    barrier(pg)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K2):
        Gd_in[0].copy_(Gh_in, non_blocking=True)
        _, mu, n, _ = ctx.step(Gd_in[0], Gd_out[0])
        Gh_out[0].copy_(Gd_out[0], non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    barrier(pg)
    ms_e2e_serial = max_over_ranks(pg, e0.elapsed_time(e1), dev)
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    done = [torch.cuda.Event(), torch.cuda.Event()]
    loaded = [torch.cuda.Event(), torch.cuda.Event()]
    barrier(pg)
    torch.cuda.synchronize()
    e0.record()
    with torch.cuda.stream(copy):
        Gd_in[0].copy_(Gh_in, non_blocking=True)
        loaded[0].record(copy)
    for i in range(K2):
        b = i % 2
        if i + 1 < K2:
            with torch.cuda.stream(copy):
                if i >= 1:
                    copy.wait_event(done[1 - b])         # step i - 1 released its buffers
                Gd_in[1 - b].copy_(Gh_in, non_blocking=True)
                loaded[1 - b].record(copy)
        comp.wait_event(loaded[b])
        _, mu, n, _ = ctx.step(Gd_in[b], Gd_out[b])
        done[b].record(comp)
        with torch.cuda.stream(copy):
            copy.wait_event(done[b])
            Gh_out[b].copy_(Gd_out[b], non_blocking=True)
    comp.wait_stream(copy)
    e1.record()
    torch.cuda.synchronize()
    barrier(pg)
    ms_e2e = max_over_ranks(pg, e0.elapsed_time(e1), dev)
    # host <-> device copy rates of this machine (one pinned copy each way, alone)
    rates = {}
    for name, dst, src in (("h2d_gbs", Gd_in[0], Gh_in), ("d2h_gbs", Gh_out[0], Gd_out[0])):
        torch.cuda.synchronize()
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        rates[name] = Gh_in.numel() * Gh_in.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    gbytes = Gh_in.numel() * Gh_in.element_size()
    r, nk, no, rho, nb = ctx.r, ctx.nk, ctx.norb, ctx.rho, ctx.nb
    hfqp = hf_qp_timing(ctx, pk)
    del ctx, Gd_in, Gd_out, Gh_out
    torch.cuda.empty_cache()

    def adjoint_timing(c):
        """One qa_gw_backward at the forward's mu (after one untimed call): the
        adjoint of a step from G0 with a seeded random cotangent of the new G."""
        G0 = c.get(qa.QA_G0).clone()
        _, mu_f, _, _ = c.step(G0, c.new_g())
        gen = torch.Generator(device=dev).manual_seed(2604222230)
        Gbar = torch.randn(c.g_shape + (2,), dtype=torch.float64, device=dev, generator=gen)
        Gbar = torch.view_as_complex(Gbar)
        c.backward(G0, mu_f, Gbar_out=Gbar)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        c.backward(G0, mu_f, Gbar_out=Gbar)
        e1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(pg, e0.elapsed_time(e1), dev)
        return {"ms": ms, "what": "qa_gw_backward (FP64, %s pair basis, mu frozen at the forward's "
                                  "value, LU factors of 1 - VP kept by its forward recompute): cotangent "
                                  "of the new G in; G_in, t(R) and V(R) cotangents out"
                                  % ("reduced" if c.reduced else "full"),
                "forward_plus_adjoint_ms": None}

    def other(prec, pairs, K, adjoint=False):
        c = qa.Context(model, prec, device=str(dev), pairs=pairs)
        ms, stg, _, _, _ = timed(c, K, 1)
        ms = max_over_ranks(pg, ms, dev)
        out = {"value": world * K / (ms / 1e3), "ms_per_step": ms / K, "steps": K,
               "pair_basis": "reduced rho=%d" % c.rho if c.reduced else "full npair=%d" % c.npair,
               "stage_ms": stg, "roofline": roofline(c, prec, stg, pk),
               "iteration_hbm_frac": iteration_bytes(c, prec) / (ms / K * 1e-3) / 1e9 / pk["hbm_gbs"]}
        if adjoint:
            out["adjoint"] = adjoint_timing(c)
            out["adjoint"]["forward_plus_adjoint_ms"] = out["ms_per_step"] + out["adjoint"]["ms"]
        del c
        torch.cuda.empty_cache()
        return out

    def timed_gpu(m):
        c = qa.Context(m, "mixed", device=str(dev))
        ms, _, _, _, _ = timed(c, 10, 3)
        del c
        torch.cuda.empty_cache()
        return ms / 10

    table1 = paper_table1(qa, wl, dev, pg, world, timed)
    fp32 = other("fp32", "auto", args.other_steps)
    full_mixed = other("mixed", "full", 2)
    fp64 = other("fp64", "full", args.fp64_steps, adjoint=not args.no_adjoint)
    fp64_red = other("fp64", "reduced", args.fp64_steps, adjoint=not args.no_adjoint)
    acc = accuracy_check(qa, wl, dev)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_block(qa, wl, dev, timed_gpu)
    ms_step = ms_mixed / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "df (double-float: FP32 pairs) storage and arithmetic; bf16-slice tensor cores for the "
                 "DLR maps; FP64 mu and density",
        "data": "synthetic: seeded five-orbital Hund-Hubbard model (SplitMix64), no dataset",
        "config": {"workload": WORKLOAD, "k_grid": [32, 32, 8], "norb": no, "npair": no * no,
                   "pair_basis": "reduced: rho=%d of %d pairs (exact; W^C = B Wt^C B^H)" % (rho, no * no)
                   if nb < no * no else "full", "dlr_rank": r, "beta": 100.0, "Lambda": 1e4, "eps": 1e-12,
                   "precision": "mixed (QA_MIXED: Sigma within 1e-7 of the FP64 oracle)",
                   "l2": "no flush: per-step working set (P, W^C: 2 x %.2f GB) is far larger than the "
                         "129 MB L2" % (r * nb * nb * nk * 16 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iteration": {"hbm_bytes": it_bytes, "hbm_frac": it_bytes / (ms_step * 1e-3) / 1e9 / pk["hbm_gbs"],
                      "mu_evals_per_step": statistics.mean(evals)},
        "stage_ms": stage_mixed,
        "accuracy": acc,
        "fp32_fast_mode": fp32,
        "mixed_full_pair_basis": full_mixed,
        "fp64": fp64,
        "fp64_reduced_pair_basis": fp64_red,
        "speedup_mixed_over_fp64": fp64["ms_per_step"] / ms_step,
        "speedup_mixed_over_fp64_reduced": fp64_red["ms_per_step"] / ms_step,
        "peaks": pk,
        "roofline": rl,
        "hf_loop_and_qp": hfqp,
        "paper_table1_workload": table1,
        "cpu_baseline": cpu,
        "e2e": {"value": world * K2 / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": gbytes,
                "d2h_bytes_per_step": gbytes + 8 + no * no * 16,
                "copies": "pinned host G in and out every step on a second stream, overlapped with "
                          "the neighbouring steps (double-buffered)",
                "serial_value": world * K2 / (ms_e2e_serial / 1e3), **rates},
        "gpu_launches": launches,
        "clocks": ck,
    }
    print(json.dumps(line))


def run_reference(args):
    """The CPU oracle as the reference arm (bounded samples, extrapolated)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import workloads as wl
    from oracle import gw, lattice
    model = wl.config(WORKLOAD)
    dlr = gw.make_dlr(model)
    rng = np.random.default_rng(0)
    nk, r, no, npair = model.nk, dlr.r, model.norb, model.npair
    G = rng.normal(size=(nk, r, no, no)) + 1j * rng.normal(size=(nk, r, no, no))
    Grefl = gw.reflected(model, dlr, G)
    Vq = lattice.V_q(model)
    Hk = lattice.H_k(model)
    # warm-up steps also measure the per-k Sigma cost and one density evaluation
    WC = np.zeros((nk, r, npair, npair), dtype=np.complex128)
    tk, td = [], []
    for i in range(max(args.warmup, 1)):
        t0 = time.perf_counter()
        gw.self_energy_at_k(model, G, WC, i % nk)
        tk.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        gw.density_from_iw(dlr, gw.g_iw(dlr, Hk, 0.0))
        td.append(time.perf_counter() - t0)
    del WC
    iters, walls = [], []
    for i in range(args.steps):
        t0 = time.perf_counter()
        P = gw.polarization_at_q(model, dlr, G, (7 * i) % nk, Grefl)
        gw.screened_interaction(Vq[(7 * i) % nk:(7 * i) % nk + 1], P[None])
        tq = time.perf_counter() - t0
        walls.append(tq)
        iters.append(nk * (tq + statistics.mean(tk)) + 45 * statistics.mean(td))
    t_iter = statistics.mean(iters)
    value = 1.0 / t_iter
    sample = ("per step: the explicit-sum FP64 oracle's bubble + DLR + W Dyson for one q-point "
              "of the 32x32x8 workload (timed), plus the per-k Sigma q-sum and one density "
              "evaluation timed in warm-up; value = one iteration extrapolated to 8192 q, 8192 k "
              "and 45 bisection steps; ms_per_step = the measured wall time of one step's sample")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3,
        "extrapolated_ms_per_iteration": t_iter * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded five-orbital Hund-Hubbard model (SplitMix64), no dataset",
        "config": {"workload": WORKLOAD, "k_grid": [32, 32, 8], "norb": no, "dlr_rank": r,
                   "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--other-steps", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
