"""Thin ctypes binding of libqeq.so (include/qeq.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Device arrays are torch CUDA tensors (float64 / int32, contiguous); the plan
owns a private CUDA stream that waits for the caller's current stream before
each call.  If the library is missing the import fails loudly: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqeq.so")

QEQ_OK, QEQ_ERR_INVALID, QEQ_ERR_NOT_PD, QEQ_ERR_NOCONV, QEQ_ERR_CUDA, QEQ_ERR_OOM, QEQ_ERR_TIMEOUT, \
    QEQ_ERR_CAPACITY = range(8)
QEQ_FP64, QEQ_MIXED = 0, 1
QEQ_WARM_COLD, QEQ_WARM_USER, QEQ_WARM_MLP = 0, 1, 2
QEQ_FLAG_NO_GRAPH = 1
QEQ_FLAG_TEST_STALL = 2
QEQ_FLAG_TWO_RHS = 4
QEQ_FLAG_SQNM = 8
QEQ_FLAG_CHECK_DD = 16
QEQ_FLAG_CHECK_FP64 = 32
QEQ_N_STAGES = 8
STAGE_NAMES = ["species_sums", "spread", "fft_z", "fft_y", "fft_x_green", "ifft_y", "ifft_z", "gather"]

EXPORTED = ["qeq_plan_create", "qeq_plan_destroy", "qeq_plan_query", "qeq_solve", "qeq_energy", "qeq_matvec",
            "qeq_profile_matvec", "qeq_status_str", "qeq_last_error", "qeq_matvec_static", "qeq_mlp_create",
            "qeq_mlp_destroy", "qeq_mlp_set_params", "qeq_mlp_get_params", "qeq_mlp_set_adam_state",
            "qeq_mlp_forward", "qeq_mlp_train_step", "qeq_features", "qeq_plan_set_warm_start", "qeq_forces",
            "qeq_embedding", "qeq_stress", "qeq_dense_create", "qeq_dense_destroy", "qeq_dense_last_error",
            "qeq_dense_assemble", "qeq_dense_invert", "qeq_dense_charges", "qeq_dense_backward",
            "qeq_dense_matrix", "qeq_dense_query"]
MLP_NFEAT, MLP_NHIDDEN, MLP_NPARAM, MLP_RCUT = 32, 64, 6400, 6.0


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("n_struct", ctypes.c_int32),
        ("atom_offsets", ctypes.POINTER(ctypes.c_int64)),
        ("cells", ctypes.POINTER(ctypes.c_double)),
        ("n_species", ctypes.c_int32),
        ("sigma", ctypes.POINTER(ctypes.c_double)),
        ("coulomb_k", ctypes.c_double),
        ("charge_tol", ctypes.c_double),
        ("ewald_tol", ctypes.c_double),
        ("r_cut", ctypes.c_double),
        ("spline_order", ctypes.c_int32),
        ("mesh_spacing", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("residual_tol", ctypes.c_double),
        ("flags", ctypes.c_int32),
        ("preconditioner", ctypes.c_int32),
        ("precond_spacing", ctypes.c_double),
        ("precond_width", ctypes.c_double),
        ("precond_scale", ctypes.c_double),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("warm_used", ctypes.c_int32),
        ("residual_inf", ctypes.c_double),
        ("residual_l2", ctypes.c_double),
        ("error_bound_l2", ctypes.c_double),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("mesh", ctypes.c_int32 * 3),
        ("spline_order", ctypes.c_int32),
        ("n_species", ctypes.c_int32),
        ("narrow_pairs", ctypes.c_int32),
        ("omega", ctypes.c_double),
        ("r_cut", ctypes.c_double),
        ("volume", ctypes.c_double),
        ("n_atoms", ctypes.c_int64),
        ("pair_capacity", ctypes.c_int64),
        ("workspace_bytes", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libqeq.so and declare its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2607_17978_b300.build`")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
    lib.qeq_plan_create.argtypes = [ctypes.POINTER(PlanDesc), vp, ctypes.POINTER(vp)]
    lib.qeq_plan_create.restype = ctypes.c_int
    lib.qeq_plan_destroy.argtypes = [vp]
    lib.qeq_plan_destroy.restype = None
    lib.qeq_plan_query.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(PlanInfo)]
    lib.qeq_plan_query.restype = ctypes.c_int
    lib.qeq_solve.argtypes = [vp, vp, vp, vp, vp, dp, ctypes.c_int32, vp, vp, ctypes.POINTER(Info)]
    lib.qeq_solve.restype = ctypes.c_int
    lib.qeq_energy.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.qeq_energy.restype = ctypes.c_int
    lib.qeq_matvec.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int32]
    lib.qeq_matvec.restype = ctypes.c_int
    lib.qeq_forces.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.qeq_forces.restype = ctypes.c_int
    lib.qeq_dense_create.argtypes = [ctypes.POINTER(PlanDesc), vp, ctypes.POINTER(vp)]
    lib.qeq_dense_create.restype = ctypes.c_int
    lib.qeq_dense_destroy.argtypes = [vp]
    lib.qeq_dense_destroy.restype = None
    lib.qeq_dense_last_error.argtypes = [vp]
    lib.qeq_dense_last_error.restype = ctypes.c_char_p
    lib.qeq_dense_assemble.argtypes = [vp, vp, vp]
    lib.qeq_dense_assemble.restype = ctypes.c_int
    lib.qeq_dense_invert.argtypes = [vp, vp]
    lib.qeq_dense_invert.restype = ctypes.c_int
    lib.qeq_dense_charges.argtypes = [vp, vp, dp, vp, vp]
    lib.qeq_dense_charges.restype = ctypes.c_int
    lib.qeq_dense_backward.argtypes = [vp, vp, vp, vp, vp]
    lib.qeq_dense_backward.restype = ctypes.c_int
    lib.qeq_dense_matrix.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp]
    lib.qeq_dense_matrix.restype = ctypes.c_int
    lib.qeq_dense_query.argtypes = [vp, ctypes.c_int32, dp, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int64)]
    lib.qeq_dense_query.restype = ctypes.c_int
    lib.qeq_stress.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.qeq_stress.restype = ctypes.c_int
    lib.qeq_embedding.argtypes = [vp, vp, vp, vp, vp]
    lib.qeq_embedding.restype = ctypes.c_int
    lib.qeq_profile_matvec.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
    lib.qeq_profile_matvec.restype = ctypes.c_int
    lib.qeq_status_str.argtypes = [ctypes.c_int]
    lib.qeq_status_str.restype = ctypes.c_char_p
    lib.qeq_last_error.argtypes = [vp]
    lib.qeq_last_error.restype = ctypes.c_char_p
    lib.qeq_matvec_static.argtypes = [dp, dp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, vp]
    lib.qeq_matvec_static.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    lib.qeq_mlp_create.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(vp)]
    lib.qeq_mlp_create.restype = ctypes.c_int
    lib.qeq_mlp_destroy.argtypes = [vp]
    lib.qeq_mlp_destroy.restype = None
    lib.qeq_mlp_set_params.argtypes = [vp, fp, fp]
    lib.qeq_mlp_set_params.restype = ctypes.c_int
    lib.qeq_mlp_get_params.argtypes = [vp, fp, fp, fp, fp, ctypes.POINTER(ctypes.c_int64)]
    lib.qeq_mlp_get_params.restype = ctypes.c_int
    lib.qeq_mlp_set_adam_state.argtypes = [vp, fp, fp, ctypes.c_int64]
    lib.qeq_mlp_set_adam_state.restype = ctypes.c_int
    lib.qeq_mlp_forward.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp]
    lib.qeq_mlp_forward.restype = ctypes.c_int
    lib.qeq_mlp_train_step.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.c_int32, vp, fp, vp]
    lib.qeq_mlp_train_step.restype = ctypes.c_int
    lib.qeq_features.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.qeq_features.restype = ctypes.c_int
    lib.qeq_plan_set_warm_start.argtypes = [vp, vp]
    lib.qeq_plan_set_warm_start.restype = ctypes.c_int
    del ip
    if path == LIB_PATH:
        _lib = lib
    return lib


class QEqError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


@dataclass
class SolveResult:
    q: "object"          # torch tensor (N,) float64, input atom order
    mu: "object"         # torch tensor (n_struct,) float64
    info: list           # list of dicts


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """A solve plan for fixed cells, atom counts and species widths."""

    def __init__(self, cells, atom_offsets, sigma, *, coulomb_k=14.3996454784, charge_tol=1e-5,
                 ewald_tol=1e-6, r_cut=8.0, spline_order=0, mesh_spacing=0.0, precision="fp64",
                 max_iter=1000, residual_tol=0.0, graph=True, device=None, preconditioner="jacobi",
                 precond_spacing=0.0, precond_width=0.0, precond_scale=0.0, test_stall=False,
                 solver="projected", check="auto"):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device or "cuda")
        cells = np.ascontiguousarray(np.asarray(cells, np.float64).reshape(-1, 9))
        offs = np.ascontiguousarray(np.asarray(atom_offsets, np.int64))
        sigma = np.ascontiguousarray(np.atleast_2d(np.asarray(sigma, np.float64)))
        self.n_struct = int(cells.shape[0])
        if sigma.shape[0] != self.n_struct:
            raise ValueError("sigma must have one row per structure")
        self.n_species = int(sigma.shape[1])
        self.n_atoms = int(offs[-1])
        self._keep = (cells, offs, sigma)
        prec = {"fp64": QEQ_FP64, "mixed": QEQ_MIXED}[precision]
        self.precision = precision
        d = PlanDesc(self.n_struct, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     cells.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.n_species,
                     sigma.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), coulomb_k, charge_tol, ewald_tol,
                     r_cut, spline_order, mesh_spacing, prec, max_iter, residual_tol,
                     (0 if graph else QEQ_FLAG_NO_GRAPH) | (QEQ_FLAG_TEST_STALL if test_stall else 0)
                     | {"projected": 0, "two_rhs": QEQ_FLAG_TWO_RHS, "sqnm": QEQ_FLAG_SQNM}[solver]
                     | {"auto": 0, "dd": QEQ_FLAG_CHECK_DD, "fp64": QEQ_FLAG_CHECK_FP64}[check],
                     {"jacobi": 0, "fourier": 1}[preconditioner],
                     precond_spacing, precond_width, precond_scale)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(device=self.device)
            h = ctypes.c_void_p()
            st = self.lib.qeq_plan_create(ctypes.byref(d), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != QEQ_OK:
            raise QEqError(st, "qeq_plan_create: " + self.lib.qeq_status_str(st).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.qeq_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st not in (QEQ_OK,):
            msg = self.lib.qeq_last_error(self.h).decode()
            raise QEqError(st, f"{what}: {self.lib.qeq_status_str(st).decode()}: {msg}")

    def _dev(self, x, dtype):
        t = self.torch.as_tensor(x, dtype=dtype, device=self.device)
        return t.contiguous()

    def query(self, s: int = 0) -> dict:
        pi = PlanInfo()
        self._check(self.lib.qeq_plan_query(self.h, s, ctypes.byref(pi)), "qeq_plan_query")
        return {"mesh": tuple(pi.mesh), "spline_order": pi.spline_order, "n_species": pi.n_species,
                "narrow_pairs": pi.narrow_pairs, "omega": pi.omega, "r_cut": pi.r_cut, "volume": pi.volume,
                "n_atoms": pi.n_atoms, "pair_capacity": pi.pair_capacity, "workspace_bytes": pi.workspace_bytes,
                "kernel_launches": pi.kernel_launches}

    def _sync_in(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def features(self, pos, species, chi, J):
        """Descriptors (n_atoms x 32 float32, the caller's atom order)."""
        torch = self.torch
        pos = self._dev(pos, torch.float64).reshape(-1, 3)
        species = self._dev(species, torch.int32)
        chi = self._dev(chi, torch.float64)
        J = self._dev(J, torch.float64)
        f = torch.empty(self.n_atoms, MLP_NFEAT, dtype=torch.float32, device=self.device)
        self._sync_in()
        self._check(self.lib.qeq_features(self.h, _ptr(pos), _ptr(species), _ptr(chi), _ptr(J), _ptr(f)),
                    "qeq_features")
        return f

    def set_warm_start(self, mlp):
        self._mlp = mlp
        self._check(self.lib.qeq_plan_set_warm_start(self.h, mlp.h if mlp is not None else None),
                    "qeq_plan_set_warm_start")

    def solve(self, pos, species, chi, J, q_tot=None, q0=None, raise_on_noconv=True, out=None, warm=None):
        torch = self.torch
        pos = self._dev(pos, torch.float64).reshape(-1, 3)
        species = self._dev(species, torch.int32)
        chi = self._dev(chi, torch.float64)
        J = self._dev(J, torch.float64)
        if q_tot is None:
            q_tot = np.zeros(self.n_struct)
        qt = np.ascontiguousarray(np.broadcast_to(np.asarray(q_tot, np.float64), (self.n_struct,)))
        q = out if out is not None else torch.empty(self.n_atoms, dtype=torch.float64, device=self.device)
        if warm == "mlp":
            warm = QEQ_WARM_MLP
        elif q0 is not None:
            q.copy_(self._dev(q0, torch.float64))
            warm = QEQ_WARM_USER
        else:
            warm = QEQ_WARM_COLD
        mu = torch.empty(self.n_struct, dtype=torch.float64, device=self.device)
        info = (Info * self.n_struct)()
        self._sync_in()
        st = self.lib.qeq_solve(self.h, _ptr(pos), _ptr(species), _ptr(chi), _ptr(J),
                                qt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), warm, _ptr(q), _ptr(mu), info)
        if st != QEQ_OK and not (st == QEQ_ERR_NOCONV and not raise_on_noconv):
            self._check(st, "qeq_solve")
        infos = [{k: getattr(i, k) for k, _ in Info._fields_} for i in info]
        return SolveResult(q, mu, infos)

    def energy(self, pos, species, chi, J, q):
        torch = self.torch
        pos = self._dev(pos, torch.float64).reshape(-1, 3)
        species = self._dev(species, torch.int32)
        chi = self._dev(chi, torch.float64)
        J = self._dev(J, torch.float64)
        q = self._dev(q, torch.float64)
        E = torch.empty(self.n_struct, dtype=torch.float64, device=self.device)
        Ee = torch.empty(self.n_struct, dtype=torch.float64, device=self.device)
        self._sync_in()
        self._check(self.lib.qeq_energy(self.h, _ptr(pos), _ptr(species), _ptr(chi), _ptr(J), _ptr(q), _ptr(E),
                                        _ptr(Ee)), "qeq_energy")
        return E, Ee

    def matvec(self, pos, species, x, J=None, fp64=False):
        torch = self.torch
        pos = self._dev(pos, torch.float64).reshape(-1, 3)
        species = self._dev(species, torch.int32)
        x = self._dev(x, torch.float64)
        Jt = self._dev(J, torch.float64) if J is not None else None
        y = torch.empty(self.n_atoms, dtype=torch.float64, device=self.device)
        self._sync_in()
        self._check(self.lib.qeq_matvec(self.h, _ptr(pos), _ptr(species), _ptr(Jt), _ptr(x), _ptr(y),
                                        1 if fp64 else 0), "qeq_matvec")
        return y

    def forces(self, pos, species, q, lam=None):
        """Electrostatic forces of the force trick (qeq_forces): N x 3, input order."""
        torch = self.torch
        pos = self._dev(pos, torch.float64).reshape(-1, 3)
        species = self._dev(species, torch.int32)
        q = self._dev(q, torch.float64)
        lt = self._dev(lam, torch.float64) if lam is not None else None
        F = torch.empty(self.n_atoms, 3, dtype=torch.float64, device=self.device)
        self._sync_in()
        self._check(self.lib.qeq_forces(self.h, _ptr(pos), _ptr(species), _ptr(q), _ptr(lt), _ptr(F)),
                    "qeq_forces")
        return F

    def stress(self, pos, species, q, lam=None):
        """Strain derivative d/d eps [(q/2 + lam)^T E q] per structure (qeq_stress): n_struct x 3 x 3."""
        torch = self.torch
        pos = self._dev(pos, torch.float64).reshape(-1, 3)
        species = self._dev(species, torch.int32)
        q = self._dev(q, torch.float64)
        lt = self._dev(lam, torch.float64) if lam is not None else None
        D = torch.empty(self.n_struct, 3, 3, dtype=torch.float64, device=self.device)
        self._sync_in()
        self._check(self.lib.qeq_stress(self.h, _ptr(pos), _ptr(species), _ptr(q), _ptr(lt), _ptr(D)),
                    "qeq_stress")
        return D

    def embedding(self, pos, species, q):
        """Element-resolved potentials (qeq_embedding): N x n_species, input order."""
        torch = self.torch
        pos = self._dev(pos, torch.float64).reshape(-1, 3)
        species = self._dev(species, torch.int32)
        q = self._dev(q, torch.float64)
        G = torch.empty(self.n_atoms, self.n_species, dtype=torch.float64, device=self.device)
        self._sync_in()
        self._check(self.lib.qeq_embedding(self.h, _ptr(pos), _ptr(species), _ptr(q), _ptr(G)), "qeq_embedding")
        return G

    def profile_matvec(self, n_rep: int = 10) -> dict:
        ms = (ctypes.c_float * QEQ_N_STAGES)()
        self._check(self.lib.qeq_profile_matvec(self.h, n_rep, ms), "qeq_profile_matvec")
        return dict(zip(STAGE_NAMES, [float(v) for v in ms]))


class Mlp:
    """Warm-start network (qeq_mlp): per-species 32 -> 64 -> 64 -> 1 on the GPU."""

    def __init__(self, n_species, max_batch=65536, device=None):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device or "cuda")
        self.n_species = int(n_species)
        self.max_batch = int(max_batch)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(device=self.device)
            st = self.lib.qeq_mlp_create(self.n_species, self.max_batch, ctypes.byref(h))
        if st != QEQ_OK:
            raise QEqError(st, "qeq_mlp_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.qeq_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f(self, a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None else None

    def set_params(self, params=None, scale=None):
        p = None if params is None else np.ascontiguousarray(params, np.float32).reshape(-1)
        sc = None if scale is None else np.ascontiguousarray(scale, np.float32).reshape(-1)
        if p is not None and p.size != self.n_species * MLP_NPARAM:
            raise ValueError("params size")
        if sc is not None and sc.size != self.n_species * 2 * MLP_NFEAT:
            raise ValueError("scale size")
        st = self.lib.qeq_mlp_set_params(self.h, self._f(p), self._f(sc))
        if st != QEQ_OK:
            raise QEqError(st, "qeq_mlp_set_params")

    def get_state(self):
        npar = self.n_species * MLP_NPARAM
        p = np.zeros(npar, np.float32)
        sc = np.zeros(self.n_species * 2 * MLP_NFEAT, np.float32)
        m = np.zeros(npar, np.float32)
        v = np.zeros(npar, np.float32)
        step = ctypes.c_int64(0)
        st = self.lib.qeq_mlp_get_params(self.h, self._f(p), self._f(sc), self._f(m), self._f(v), ctypes.byref(step))
        if st != QEQ_OK:
            raise QEqError(st, "qeq_mlp_get_params")
        return {"params": p, "scale": sc, "adam_m": m, "adam_v": v, "step": int(step.value)}

    def set_adam_state(self, m, v, step):
        m = np.ascontiguousarray(m, np.float32)
        v = np.ascontiguousarray(v, np.float32)
        st = self.lib.qeq_mlp_set_adam_state(self.h, self._f(m), self._f(v), int(step))
        if st != QEQ_OK:
            raise QEqError(st, "qeq_mlp_set_adam_state")

    def forward(self, feat, species):
        torch = self.torch
        feat = torch.as_tensor(feat, dtype=torch.float32, device=self.device).contiguous()
        species = torch.as_tensor(species, dtype=torch.int32, device=self.device).contiguous()
        out = torch.empty(feat.shape[0], dtype=torch.float32, device=self.device)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        st = self.lib.qeq_mlp_forward(self.h, _ptr(feat), _ptr(species), feat.shape[0], _ptr(out),
                                      ctypes.c_void_p(self.stream.cuda_stream))
        if st != QEQ_OK:
            raise QEqError(st, "qeq_mlp_forward")
        return out

    def train_step(self, feat, species, target, lr=1e-3, apply=True, want_grad=False):
        torch = self.torch
        grad = torch.empty(self.n_species * MLP_NPARAM, dtype=torch.float32, device=self.device) if want_grad else None
        loss = ctypes.c_float(0.0)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        st = self.lib.qeq_mlp_train_step(self.h, _ptr(feat), _ptr(species), _ptr(target), feat.shape[0], float(lr),
                                         1 if apply else 0, _ptr(grad), ctypes.byref(loss),
                                         ctypes.c_void_p(self.stream.cuda_stream))
        if st != QEQ_OK:
            raise QEqError(st, "qeq_mlp_train_step")
        return float(loss.value), grad


def matvec_static(cell, sigma_s, pos, species, x, J=None, *, coulomb_k=14.3996454784, ewald_tol=1e-6,
                  r_cut=8.0, stream=None, device=None):
    """FP64 matvec of one small cell through qeq_matvec_static (no device allocation in the library).

    Inputs are converted to contiguous float64 / int32 tensors on the target
    device and their sizes checked against n = len(x) before the call; the
    output tensor is allocated here (torch), the library itself allocates
    nothing.  The call runs on ``stream`` (default: torch's current stream of
    that device), so it is ordered after the caller's earlier work there.
    """
    import torch
    lib = load_library()
    dev = torch.device(device) if device is not None else (x.device if isinstance(x, torch.Tensor) else
                                                           torch.device("cuda"))
    if dev.type != "cuda":
        raise QEqError(QEQ_ERR_INVALID, "qeq_matvec_static needs CUDA tensors")

    def _as(t, dtype):
        return torch.as_tensor(t, dtype=dtype, device=dev).contiguous()

    x = _as(x, torch.float64).reshape(-1)
    pos = _as(pos, torch.float64).reshape(-1)
    species = _as(species, torch.int32).reshape(-1)
    J = _as(J, torch.float64).reshape(-1) if J is not None else None
    n = int(x.numel())
    if pos.numel() != 3 * n or species.numel() != n or (J is not None and J.numel() != n):
        raise QEqError(QEQ_ERR_INVALID, f"qeq_matvec_static: pos must hold 3n, species and J n entries (n = {n})")
    cell = np.ascontiguousarray(np.asarray(cell, np.float64).reshape(9))
    sig = np.ascontiguousarray(np.asarray(sigma_s, np.float64).reshape(-1))
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        st = lib.qeq_matvec_static(cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(sig), n, _ptr(pos),
                                   _ptr(species), _ptr(J), _ptr(x), _ptr(y), coulomb_k, ewald_tol, r_cut,
                                   ctypes.c_void_p(stream.cuda_stream))
    if st != QEQ_OK:
        raise QEqError(st, "qeq_matvec_static: " + lib.qeq_status_str(st).decode())
    return y


class Dense:
    """4G charge training on cached dense matrices (qeq_dense_*): E per structure once, the
    bordered inverse per hardness, charges and their backward pass as matrix-vector products."""

    def __init__(self, cells, atom_offsets, sigma, *, coulomb_k=14.3996454784, ewald_tol=0.0, device=None,
                 precision="fp64"):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device or "cuda")
        cells = np.ascontiguousarray(np.asarray(cells, np.float64).reshape(-1, 9))
        offs = np.ascontiguousarray(np.asarray(atom_offsets, np.int64))
        sigma = np.ascontiguousarray(np.atleast_2d(np.asarray(sigma, np.float64)))
        self.n_struct = int(cells.shape[0])
        if sigma.shape[0] != self.n_struct:
            raise ValueError("sigma must have one row per structure")
        self.n_species = int(sigma.shape[1])
        self.n_atoms = int(offs[-1])
        self.offsets = offs
        self._keep = (cells, offs, sigma)
        d = PlanDesc(self.n_struct, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                     cells.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.n_species,
                     sigma.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), coulomb_k, 0.0, ewald_tol,
                     0.0, 0, 0.0, {"fp64": QEQ_FP64, "mixed": QEQ_MIXED}[precision], 0, 0.0, 0, 0, 0.0, 0.0, 0.0)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(device=self.device)
            h = ctypes.c_void_p()
            st = self.lib.qeq_dense_create(ctypes.byref(d), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != QEQ_OK:
            raise QEqError(st, "qeq_dense_create: " + self.lib.qeq_status_str(st).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.torch.cuda.synchronize(self.device)
            self.lib.qeq_dense_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, x, dtype):
        return self.torch.as_tensor(x, dtype=dtype, device=self.device).contiguous()

    def _sync_in(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _sync_out(self):
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _check(self, st, what):
        if st != QEQ_OK:
            msg = self.lib.qeq_dense_last_error(self.h).decode()
            raise QEqError(st, f"{what}: {self.lib.qeq_status_str(st).decode()} ({msg})")

    def assemble(self, pos, species):
        torch = self.torch
        self._pos = self._dev(pos, torch.float64).reshape(-1, 3)
        self._spc = self._dev(species, torch.int32)
        self._sync_in()
        self._check(self.lib.qeq_dense_assemble(self.h, _ptr(self._pos), _ptr(self._spc)), "qeq_dense_assemble")

    def invert(self, J):
        self._J = self._dev(J, self.torch.float64)
        self._sync_in()
        self._check(self.lib.qeq_dense_invert(self.h, _ptr(self._J)), "qeq_dense_invert")

    def charges(self, chi, q_tot=None):
        torch = self.torch
        chi = self._dev(chi, torch.float64)
        qt = np.zeros(self.n_struct) if q_tot is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(q_tot, np.float64), (self.n_struct,)))
        q = torch.empty(self.n_atoms, dtype=torch.float64, device=self.device)
        mu = torch.empty(self.n_struct, dtype=torch.float64, device=self.device)
        self._sync_in()
        self._check(self.lib.qeq_dense_charges(self.h, _ptr(chi), qt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               _ptr(q), _ptr(mu)), "qeq_dense_charges")
        self._sync_out()
        return q, mu

    def backward(self, q, gq):
        torch = self.torch
        q = self._dev(q, torch.float64)
        gq = self._dev(gq, torch.float64)
        gchi = torch.empty(self.n_atoms, dtype=torch.float64, device=self.device)
        gJ = torch.empty(self.n_atoms, dtype=torch.float64, device=self.device)
        self._sync_in()
        self._check(self.lib.qeq_dense_backward(self.h, _ptr(q), _ptr(gq), _ptr(gchi), _ptr(gJ)), "qeq_dense_backward")
        self._sync_out()
        return gchi, gJ

    def matrix(self, s, which=0):
        n = int(self.offsets[s + 1] - self.offsets[s]) + (1 if which else 0)
        out = self.torch.empty(n, n, dtype=self.torch.float64, device=self.device)
        self._check(self.lib.qeq_dense_matrix(self.h, int(s), int(which), _ptr(out)), "qeq_dense_matrix")
        self._sync_out()
        return out

    def query(self, s=0):
        om, ng, nl = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int64()
        self._check(self.lib.qeq_dense_query(self.h, int(s), ctypes.byref(om), ctypes.byref(ng), ctypes.byref(nl)),
                    "qeq_dense_query")
        return {"omega": om.value, "n_g": ng.value, "kernel_launches": nl.value}


def dense_for_structures(structs, **kw) -> Dense:
    """Dense charge-training handle for a list of ``synth.Structure``."""
    ns = max(s.n_species for s in structs)
    cells = np.stack([s.cell for s in structs]).reshape(-1, 9)
    offs = np.concatenate([[0], np.cumsum([s.n for s in structs])]).astype(np.int64)
    sig = np.zeros((len(structs), ns))
    for i, s in enumerate(structs):
        sig[i, :s.n_species] = s.sigma_s
    return Dense(cells, offs, sig, **kw)


def plan_for_structures(structs, **kw) -> Plan:
    """Plan for a list of ``synth.Structure`` (same species-table width)."""
    ns = max(s.n_species for s in structs)
    cells = np.stack([s.cell for s in structs]).reshape(-1, 9)
    offs = np.concatenate([[0], np.cumsum([s.n for s in structs])]).astype(np.int64)
    sig = np.zeros((len(structs), ns))          # trailing zeros: species absent from that structure
    for i, s in enumerate(structs):
        sig[i, :s.n_species] = s.sigma_s
    return Plan(cells, offs, sig, **kw)


def pack(structs):
    """Concatenate per-structure atom arrays (positions, species, chi, J, q_tot)."""
    pos = np.concatenate([s.pos for s in structs])
    spc = np.concatenate([s.species for s in structs]).astype(np.int32)
    chi = np.concatenate([s.chi for s in structs])
    J = np.concatenate([s.J for s in structs])
    qt = np.array([s.q_tot for s in structs])
    return pos, spc, chi, J, qt
