"""ctypes binding of libqa (argument marshalling only).

Every step of the GW iteration runs in the CUDA kernels behind the C ABI in
include/qa.h; this module converts Python/numpy/torch arguments to the
ABI's plain pointers and sizes and raises on a non-zero status.  PyTorch
provides the device memory (the context workspace and the G arrays) and the
CUDA stream.  There is no CPU fallback: without the library or a GPU the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqa.so")

QA_FP64, QA_MIXED, QA_FP32 = 0, 1, 2
PRECISIONS = {"fp64": QA_FP64, "mixed": QA_MIXED, "fp32": QA_FP32}
QA_PAIRS_AUTO, QA_PAIRS_FULL, QA_PAIRS_REDUCED = 0, 1, 2
QA_P_QNU, QA_WC_RTAU, QA_SIGC_KTAU, QA_SIGC_KIW, QA_SIGHF_K, QA_G0, QA_HK, QA_MU0 = range(1, 9)

EXPORTED = ["qa_create", "qa_workspace_size", "qa_bind", "qa_get_grid", "qa_get_plan",
            "qa_get_sizes", "qa_gw_step", "qa_density", "qa_density_static", "qa_get",
            "qa_set_timing", "qa_set_mu", "qa_set_params", "qa_gw_backward", "qa_set_pair_basis",
            "qa_get_pair_basis", "qa_hf_solve", "qa_qp", "qa_destroy", "qa_strerror",
            "qa_fma_probe", "qa_set_wait_limit", "qa_free_energy", "qa_free_energy_backward"]

STAGES = ["hartree_fock", "g_to_R", "bubble", "fft_R_to_q", "dlr_tau_to_nu", "dyson_w",
          "dlr_nu_to_tau", "fft_q_to_R", "sigma", "sigma_to_k_iw", "mu_search", "dyson_g"]


def fma_rate(precision: str, iters: int = 4096, reps: int = 3):
    """Measured FMA rate of the current GPU (TFLOP/s, 2 flops per FMA) from
    qa_fma_probe: the best of `reps` CUDA-event-timed launches after one warm-up."""
    import torch
    L = load()
    prec = PRECISIONS[precision]
    n, flops = C.c_longlong(), C.c_double()
    _check(L.qa_fma_probe(prec, iters, None, C.byref(n), C.byref(flops), None), "qa_fma_probe")
    out = torch.empty(n.value, dtype=torch.float64 if prec == QA_FP64 else torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    best = None
    for rep in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _check(L.qa_fma_probe(prec, iters, out.data_ptr(), C.byref(n), C.byref(flops), stream), "qa_fma_probe")
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if rep > 0:
            best = ms if best is None else min(best, ms)
    return flops.value / (best * 1e-3) / 1e12, best


class QAError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (where, strerror(status), status))


class Lattice(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("norb", C.c_int), ("nspin", C.c_int)]


class Hoppings(C.Structure):
    _fields_ = [("nR", C.c_int), ("R", C.POINTER(C.c_int)), ("t", C.POINTER(C.c_double)),
                ("eps", C.POINTER(C.c_double))]


class Interaction(C.Structure):
    _fields_ = [("nR", C.c_int), ("R", C.POINTER(C.c_int)), ("V", C.POINTER(C.c_double))]


class StepStats(C.Structure):
    _fields_ = [("mu", C.c_double), ("N", C.c_double), ("mu_evals", C.c_int),
                ("status", C.c_int), ("first_bad", C.c_longlong), ("launches", C.c_int),
                ("stage_ms", C.c_float * 16)]


_lib = None


def load(path: str = None):
    """Load libqa.so and declare the ABI; raises if it was not built.  The
    environment variable QA_LIB names another build of the same ABI (the
    bounds-checked libqa_checked.so), read at the first load of a process."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("QA_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libqa.so not found at %s: run paper_2604_22223_gb300.build()" % path)
    L = C.CDLL(path)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    L.qa_create.argtypes = [C.POINTER(Lattice), C.POINTER(Hoppings), C.POINTER(Interaction), d, d,
                            d, d, i, C.POINTER(vp)]
    L.qa_workspace_size.argtypes = [vp, C.POINTER(sz)]
    L.qa_bind.argtypes = [vp, vp, sz, vp]
    L.qa_get_grid.argtypes = [vp, C.POINTER(i), vp, vp, vp, vp]
    L.qa_get_plan.argtypes = [vp, vp, vp, vp, vp]
    L.qa_get_sizes.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i)]
    L.qa_gw_step.argtypes = [vp, vp, vp, C.POINTER(d), vp, C.POINTER(StepStats), vp]
    L.qa_density.argtypes = [vp, vp, vp, C.POINTER(d), vp]
    L.qa_density_static.argtypes = [vp, vp, vp, C.POINTER(d), vp]
    L.qa_get.argtypes = [vp, i, vp, sz, vp]
    L.qa_set_timing.argtypes = [vp, i]
    L.qa_set_mu.argtypes = [vp, i, d]
    L.qa_set_params.argtypes = [vp, C.POINTER(Hoppings), C.POINTER(Interaction), vp]
    L.qa_gw_backward.argtypes = [vp, vp, d, vp, vp, vp, vp, vp, vp, vp]
    L.qa_set_pair_basis.argtypes = [vp, i]
    L.qa_get_pair_basis.argtypes = [vp, C.POINTER(i), C.POINTER(i), vp]
    L.qa_hf_solve.argtypes = [vp, i, d, d, vp, C.POINTER(d), C.POINTER(i), C.POINTER(d), vp, vp]
    L.qa_qp.argtypes = [vp, vp, vp, vp, vp, vp]
    L.qa_fma_probe.argtypes = [i, i, vp, C.POINTER(C.c_longlong), C.POINTER(d), vp]
    L.qa_set_wait_limit.argtypes = [vp, C.c_longlong]
    L.qa_free_energy.argtypes = [vp, vp, d, i, C.POINTER(d), vp, vp]
    L.qa_free_energy_backward.argtypes = [vp, vp, d, i, d, vp, vp, vp, vp]
    L.qa_destroy.argtypes = [vp]
    L.qa_destroy.restype = None
    L.qa_strerror.argtypes = [i]
    L.qa_strerror.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("qa_destroy", "qa_strerror"):
            getattr(L, name).restype = i
    _lib = L
    return L


def strerror(status: int) -> str:
    try:
        return load().qa_strerror(status).decode()
    except Exception:  # noqa: BLE001 - message only
        return "status %d" % status


def _check(status: int, where: str):
    if status != 0:
        raise QAError(status, where)


def _as(arr, dtype):
    return np.ascontiguousarray(arr, dtype=dtype)


class Problem:
    """Host-side problem handle (qa_create): validation, DLR grid and FFT plans.

    `model` provides n, norb, s_spin, hop_R, hop_t, eps, V_R, V, beta, Lambda,
    eps_dlr and filling (see workloads.Model).  `pairs` selects the basis of
    the big tensors: "auto" (reduced on the mixed and FP32 paths), "full" or
    "reduced" (include/qa.h, qa_set_pair_basis).  `precision`: "fp64",
    "mixed" (double-float storage, FP32-based arithmetic, ~1e-9 of FP64) or
    "fp32" (complex64 storage, the fast mode).  No GPU is touched.
    """

    def __init__(self, model, precision: str = "fp64", pairs: str = "auto"):
        L = load()
        self.model = model
        self.precision = PRECISIONS[precision]
        self._keep = []
        lat = Lattice((C.c_int * 3)(*[int(v) for v in model.n]), int(model.norb), int(model.s_spin))
        hop, inter = self._structs(model)
        ctx = C.c_void_p()
        _check(L.qa_create(C.byref(lat), C.byref(hop), C.byref(inter), float(model.beta),
                           float(model.Lambda), float(model.eps_dlr), float(model.filling),
                           self.precision, C.byref(ctx)), "qa_create")
        self.ctx = ctx
        mode = {"auto": QA_PAIRS_AUTO, "full": QA_PAIRS_FULL, "reduced": QA_PAIRS_REDUCED}[pairs]
        _check(L.qa_set_pair_basis(ctx, mode), "qa_set_pair_basis")
        nk, no, r = C.c_int(), C.c_int(), C.c_int()
        _check(L.qa_get_sizes(ctx, C.byref(nk), C.byref(no), C.byref(r)), "qa_get_sizes")
        self.nk, self.norb, self.r = nk.value, no.value, r.value
        self.npair = self.norb * self.norb
        self.rho, self.reduced, self.basis = self.pair_basis()
        self.nb = self.rho if self.reduced else self.npair

    def pair_basis(self):
        """(rho, reduced basis in use, B [npair, rho] complex128)."""
        rho, act = C.c_int(), C.c_int()
        _check(load().qa_get_pair_basis(self.ctx, C.byref(rho), C.byref(act), None), "qa_get_pair_basis")
        B = np.zeros(2 * self.npair * max(rho.value, 1))
        _check(load().qa_get_pair_basis(self.ctx, None, None, B.ctypes.data), "qa_get_pair_basis")
        B = B.view(np.complex128)[:self.npair * rho.value].reshape(self.npair, rho.value)
        return rho.value, bool(act.value), B

    def _structs(self, model):
        hR = _as(model.hop_R, np.int32)
        ht = _as(np.asarray(model.hop_t, dtype=np.complex128).view(np.float64), np.float64)
        he = _as(model.eps, np.float64)
        vR = _as(model.V_R, np.int32)
        vV = _as(np.asarray(model.V, dtype=np.complex128).view(np.float64), np.float64)
        self._keep = [hR, ht, he, vR, vV]
        hop = Hoppings(len(hR), hR.ctypes.data_as(C.POINTER(C.c_int)),
                       ht.ctypes.data_as(C.POINTER(C.c_double)),
                       he.ctypes.data_as(C.POINTER(C.c_double)))
        inter = Interaction(len(vR), vR.ctypes.data_as(C.POINTER(C.c_int)),
                            vV.ctypes.data_as(C.POINTER(C.c_double)))
        return hop, inter

    def grid(self) -> dict:
        r = self.r
        x = np.zeros(r)
        t = np.zeros(r)
        nf = np.zeros(r, np.int32)
        mb = np.zeros(r, np.int32)
        rr = C.c_int()
        _check(load().qa_get_grid(self.ctx, C.byref(rr), x.ctypes.data, t.ctypes.data,
                                  nf.ctypes.data, mb.ctypes.data), "qa_get_grid")
        return {"r": rr.value, "x": x, "t": t, "nf": nf, "mb": mb}

    def plan(self) -> dict:
        n = [int(v) for v in self.model.n]
        mR = np.zeros(self.nk, np.int32)
        pos = np.zeros(sum(n), np.int32)
        nfac = np.zeros(3, np.int32)
        fac = np.zeros((3, 16), np.int32)
        _check(load().qa_get_plan(self.ctx, mR.ctypes.data, pos.ctypes.data, nfac.ctypes.data,
                                  fac.ctypes.data), "qa_get_plan")
        return {"minus_R": mR, "pos": pos, "nfac": nfac, "fac": fac}

    def workspace_size(self) -> int:
        b = C.c_size_t()
        _check(load().qa_workspace_size(self.ctx, C.byref(b)), "qa_workspace_size")
        return b.value

    def close(self):
        if getattr(self, "ctx", None):
            load().qa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Context(Problem):
    """A bound context: Problem + device workspace (torch) + G0 (qa_bind)."""

    def __init__(self, model, precision: str = "fp64", device: str = "cuda", pairs: str = "auto"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libqa needs a CUDA GPU; no CPU fallback exists")
        super().__init__(model, precision, pairs)
        self.torch = torch
        self.device = torch.device(device)
        nbytes = self.workspace_size()
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        _check(load().qa_bind(self.ctx, self.workspace.data_ptr(), nbytes, self._stream()), "qa_bind")

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    @property
    def g_shape(self):
        return (self.r, self.norb, self.norb, self.nk)

    def new_g(self):
        return self.torch.empty(self.g_shape, dtype=self.torch.complex128, device=self.device)

    def set_wait_limit(self, polls=None):
        """Poll budget of the tensor-core kernels' pipeline waits (None: default)."""
        _check(load().qa_set_wait_limit(self.ctx, -1 if polls is None else int(polls)), "qa_set_wait_limit")

    def step(self, G_in=None, G_out=None, timing: bool = False, check: bool = True):
        """One GW iteration; returns (G_out, mu, n_local [norb, norb] complex, stats dict).
        check=False returns a failing status in stats["call_status"] instead of raising."""
        L = load()
        if G_out is None:
            G_out = self.new_g()
        for G in (G_in, G_out):
            if G is not None:
                assert G.dtype == self.torch.complex128 and G.is_contiguous() and tuple(G.shape) == self.g_shape
        _check(L.qa_set_timing(self.ctx, int(timing)), "qa_set_timing")
        mu = C.c_double()
        n = np.zeros(2 * self.norb * self.norb)
        st = StepStats()
        status = L.qa_gw_step(self.ctx, None if G_in is None else G_in.data_ptr(), G_out.data_ptr(),
                              C.byref(mu), n.ctypes.data, C.byref(st), self._stream())
        if check:
            _check(status, "qa_gw_step")
        stats = {"mu": st.mu, "N": st.N, "mu_evals": st.mu_evals, "status": st.status,
                 "first_bad": st.first_bad, "launches": st.launches, "call_status": status}
        if timing:
            stats["stage_ms"] = dict(zip(STAGES, list(st.stage_ms)[:len(STAGES)]))
        return G_out, mu.value, n.view(np.complex128).reshape(self.norb, self.norb), stats

    def set_mu(self, mu=None):
        """Hold mu fixed at `mu` for later steps (None: search again)."""
        _check(load().qa_set_mu(self.ctx, 0 if mu is None else 1, 0.0 if mu is None else float(mu)),
               "qa_set_mu")

    def set_params(self, model):
        """Replace t(R), eps and V(R) (same R lists as at creation)."""
        hop, inter = self._structs(model)
        _check(load().qa_set_params(self.ctx, C.byref(hop), C.byref(inter), self._stream()),
               "qa_set_params")
        self.model = model

    def backward(self, G_in, mu, Gbar_out=None, Sigbar=None, nbar=None, want_gin=True):
        """Adjoint of one step at fixed mu; returns (Gbar_in, grad_t, grad_V)."""
        no, npair = self.norb, self.npair
        nH, nV = len(self.model.hop_R), len(self.model.V_R)
        gt = np.zeros(2 * nH * no * no)
        gV = np.zeros(2 * max(nV, 1) * npair * npair)
        Gb = self.new_g() if want_gin else None
        nb = None if nbar is None else np.ascontiguousarray(np.asarray(nbar, np.complex128)).view(np.float64)
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(load().qa_gw_backward(self.ctx, ptr(G_in), float(mu), ptr(Gbar_out), ptr(Sigbar),
                                     None if nb is None else nb.ctypes.data, ptr(Gb), gt.ctypes.data,
                                     gV.ctypes.data, self._stream()), "qa_gw_backward")
        return (Gb, gt.view(np.complex128).reshape(nH, no, no),
                gV.view(np.complex128)[:nV * npair * npair].reshape(nV, npair, npair))

    def free_energy(self, G_in, mu, M):
        """GW grand potential of G_in at fixed mu, Matsubara cutoff M (qa_free_energy):
        (Omega, {omega_hf, omega_dc, omega_g, omega_w})."""
        om = C.c_double()
        parts = np.zeros(4)
        _check(load().qa_free_energy(self.ctx, None if G_in is None else G_in.data_ptr(), float(mu), int(M),
                                     C.byref(om), parts.ctypes.data, self._stream()), "qa_free_energy")
        return om.value, dict(zip(("omega_hf", "omega_dc", "omega_g", "omega_w"), parts.tolist()))

    def free_energy_backward(self, G_in, mu, M, omega_bar=1.0, want_gin=True):
        """Gradient of omega_bar * Omega (qa_free_energy_backward): (Gbar_in, grad_t, grad_V)."""
        no, npair = self.norb, self.npair
        nH, nV = len(self.model.hop_R), len(self.model.V_R)
        gt = np.zeros(2 * nH * no * no)
        gV = np.zeros(2 * max(nV, 1) * npair * npair)
        Gb = self.new_g() if want_gin else None
        _check(load().qa_free_energy_backward(self.ctx, None if G_in is None else G_in.data_ptr(), float(mu),
                                              int(M), float(omega_bar), None if Gb is None else Gb.data_ptr(),
                                              gt.ctypes.data, gV.ctypes.data, self._stream()),
               "qa_free_energy_backward")
        return (Gb, gt.view(np.complex128).reshape(nH, no, no),
                gV.view(np.complex128)[:nV * npair * npair].reshape(nV, npair, npair))

    def hf_solve(self, max_iter: int = 500, tol: float = 1e-10, mix: float = 1.0, G_out=None,
                 check: bool = True):
        """Self-consistent Hartree-Fock; returns (G_HF, mu, n_local, iters, resid, status).
        check=False returns QA_ENOCONV as the status instead of raising."""
        if G_out is None:
            G_out = self.new_g()
        mu, it, res = C.c_double(), C.c_int(), C.c_double()
        n = np.zeros(2 * self.norb * self.norb)
        status = load().qa_hf_solve(self.ctx, int(max_iter), float(tol), float(mix), G_out.data_ptr(),
                                    C.byref(mu), C.byref(it), C.byref(res), n.ctypes.data,
                                    self._stream())
        if check or status != 4:
            _check(status, "qa_hf_solve")
        return (G_out, mu.value, n.view(np.complex128).reshape(self.norb, self.norb), it.value,
                res.value, status)

    def qp(self):
        """Quasiparticle quantities of the current self-energy: dict of device
        tensors Z, sig0, Hqp ([N_k, norb, norb] complex128) and eps ([N_k, norb])."""
        torch = self.torch
        nk, no = self.nk, self.norb
        out = {k: torch.empty((nk, no, no), dtype=torch.complex128, device=self.device)
               for k in ("Z", "sig0", "Hqp")}
        out["eps"] = torch.empty((nk, no), dtype=torch.float64, device=self.device)
        _check(load().qa_qp(self.ctx, out["Z"].data_ptr(), out["sig0"].data_ptr(),
                            out["Hqp"].data_ptr(), out["eps"].data_ptr(), self._stream()), "qa_qp")
        return out

    def density(self, G):
        n = np.zeros(2 * self.norb * self.norb)
        N = C.c_double()
        _check(load().qa_density(self.ctx, G.data_ptr(), n.ctypes.data, C.byref(N), self._stream()),
               "qa_density")
        return n.view(np.complex128).reshape(self.norb, self.norb), N.value

    def get(self, which: int):
        """Copy an intermediate into a new device tensor (shape per include/qa.h;
        the big tensors are [r][nb][nb][N_k], nb = rho on the reduced basis)."""
        torch = self.torch
        r, no, np_, nk = self.r, self.norb, self.nb, self.nk
        big_dt = {QA_FP64: torch.complex128, QA_MIXED: "df", QA_FP32: torch.complex64}[self.precision]
        shapes = {QA_P_QNU: ((r, np_, np_, nk), big_dt), QA_WC_RTAU: ((r, np_, np_, nk), big_dt),
                  QA_SIGC_KTAU: ((r, no, no, nk), big_dt), QA_SIGC_KIW: ((r, no, no, nk), big_dt),
                  QA_SIGHF_K: ((nk, no, no), torch.complex128),
                  QA_G0: ((r, no, no, nk), torch.complex128), QA_HK: ((nk, no, no), torch.complex128)}
        if which == QA_MU0:
            v = C.c_double()
            _check(load().qa_get(self.ctx, QA_MU0, C.addressof(v), 8, self._stream()), "qa_get")
            return v.value
        shape, dt = shapes[which]
        # double-float complex arrives as four floats (re.hi, re.lo, im.hi, im.lo)
        raw = torch.empty(shape + (4,), dtype=torch.float32, device=self.device) if dt == "df" else \
            torch.empty(shape, dtype=dt, device=self.device)
        _check(load().qa_get(self.ctx, which, raw.data_ptr(), raw.numel() * raw.element_size(),
                             self._stream()), "qa_get")
        if dt == "df":
            d = raw.double()
            return torch.complex(d[..., 0] + d[..., 1], d[..., 2] + d[..., 3])
        return raw
