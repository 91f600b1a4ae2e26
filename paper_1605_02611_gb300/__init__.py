"""Thin ctypes binding of libgbdmrg.so (C-ABI declared in include/gbdmrg.h).

Argument marshalling only: every step of the DMRG hot path runs in the CUDA
library.  Importing works without a GPU; using a context needs the built
library and a CUDA device, and fails loudly otherwise (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbdmrg.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ETIMEOUT", 6: "EIO",
          7: "ESMALL", 8: "ESTATE"}

# exported symbol -> (restype, argtypes)
_P = C.c_void_p
_I32 = C.c_int32
_PI32 = C.POINTER(C.c_int32)
_PI64 = C.POINTER(C.c_int64)
_PD = C.POINTER(C.c_double)
_PF = C.POINTER(C.c_float)


class Problem(C.Structure):
    _fields_ = [("K", C.c_int32), ("N", C.c_int32), ("two_sz", C.c_int32),
                ("h1", _PD), ("eri", _PD), ("ecore", C.c_double)]


class Schedule(C.Structure):
    _fields_ = [("nsweeps", C.c_int32), ("M", _PI32), ("dav_tol", _PD), ("dav_max_iter", C.c_int32),
                ("precision", C.c_int32)]


SIGNATURES = {
    "gbdmrg_create": (C.c_int, [C.POINTER(Problem), _P, C.POINTER(_P)]),
    "gbdmrg_destroy": (None, [_P]),
    "gbdmrg_last_error": (C.c_char_p, [_P]),
    "gbdmrg_mpo_build_host": (C.c_int, [C.POINTER(Problem), _PI32, _PD]),
    "gbdmrg_mpo_bond_dims": (C.c_int, [_P, _PI32]),
    "gbdmrg_mpo_dense": (C.c_int, [_P, _PD]),
    "gbdmrg_set_mps": (C.c_int, [_P, _I32, _I32, _I32, _PI32, _PI32, _PD]),
    "gbdmrg_get_mps": (C.c_int, [_P, _I32, _PI32, _PI32, _PD]),
    "gbdmrg_get_bond": (C.c_int, [_P, _I32, _PI32, _PI32]),
    "gbdmrg_set_precision": (C.c_int, [_P, _I32]),
    "gbdmrg_prepare": (C.c_int, [_P, _I32]),
    "gbdmrg_keep_host_plans": (C.c_int, [_P, _I32]),
    "gbdmrg_set_chunk_budget": (C.c_int, [_P, _I32]),
    "gbdmrg_batch_create": (C.c_int, [_I32, C.POINTER(_P), C.POINTER(_P)]),
    "gbdmrg_batch_sigma": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), _I32, _PD, _PD]),
    "gbdmrg_batch_last_error": (C.c_char_p, [_P]),
    "gbdmrg_batch_destroy": (None, [_P]),
    "gbdmrg_set_split": (C.c_int, [_P, C.c_double]),
    "gbdmrg_get_plan_params": (C.c_int, [_P, _PD, _PI32]),
    "gbdmrg_set_stage1_stacked": (C.c_int, [_P, _I32]),
    "gbdmrg_set_tma_budget": (C.c_int, [_P, C.c_int64]),
    "gbdmrg_plan_stats": (C.c_int, [_P, _PD]),
    "gbdmrg_set_refinement": (C.c_int, [_P, _I32, _I32]),
    "gbdmrg_set_env_precision": (C.c_int, [_P, _I32]),
    "gbdmrg_set_tc_combos": (C.c_int, [_P, _I32, C.c_int64]),
    "gbdmrg_autotune": (C.c_int, [_I32, C.POINTER(_P), _I32, _PD, _I32, _PI32, _I32, _PD, _PD, _PI32]),
    "gbdmrg_plan": (C.c_int, [_P, _I32]),
    "gbdmrg_psi_layout": (C.c_int, [_P, _PI64, _PI64, _PI64]),
    "gbdmrg_sigma": (C.c_int, [_P, _P, _P, _I32, _PD]),
    "gbdmrg_diag": (C.c_int, [_P, _P, _I32]),
    "gbdmrg_diag_noalloc": (C.c_int, [_P, _P]),
    "gbdmrg_sigma_timing": (C.c_int, [_P, _I32, _P, _P, _PD]),
    "gbdmrg_step": (C.c_int, [_P, _I32, _I32, _I32, C.c_double, _I32, _P, _P, _I32, _PD, _PD, _PI32]),
    "gbdmrg_counters": (C.c_int, [_P, _PD, _PD, _PI64, _PD]),
    "gbdmrg_kernel_launches": (C.c_int64, []),
    "gbdmrg_gemm_bf16_selftest": (C.c_int, [_PI64, _I32, _PI64, _I32, _P]),
    "gbdmrg_phase_times": (C.c_int, [_P, _PD]),
    "gbdmrg_phase_flops": (C.c_int, [_P, _PD]),
    "gbdmrg_sigma_flops_host": (C.c_int, [C.POINTER(Problem), _I32, _I32, _PI32, _I32, _PI32, _PD]),
    "gbdmrg_run": (C.c_int, [_P, C.POINTER(Schedule), _PD, _PD]),
    "gbdmrg_run_stats": (C.c_int, [_P, _PD, _PD, _PD, _PI32]),
    "gbdmrg_expectation": (C.c_int, [_P, _PD]),
    "gbdmrg_save": (C.c_int, [_P, C.c_char_p]),
    "gbdmrg_load": (C.c_int, [_P, C.c_char_p]),
    "gbdmrg_mlp_nparams": (C.c_int64, []),
    "gbdmrg_mlp_create": (C.c_int, [C.c_uint64, _P, C.POINTER(_P)]),
    "gbdmrg_mlp_destroy": (None, [_P]),
    "gbdmrg_mlp_last_error": (C.c_char_p, [_P]),
    "gbdmrg_mlp_set_params": (C.c_int, [_P, _PF]),
    "gbdmrg_mlp_get_params": (C.c_int, [_P, _PF]),
    "gbdmrg_mlp_forward": (C.c_int, [_P, _P, C.c_int64, _P, _I32, _I32]),
    "gbdmrg_mlp_loss_grad": (C.c_int, [_P, _P, _P, _P, C.c_int64, _I32, _PF, _PD]),
    "gbdmrg_mlp_train": (C.c_int, [_P, _P, _P, _P, C.c_int64, _I32, _I32, _I32, C.c_float, C.c_uint64, _PD, _PD]),
    "gbdmrg_set_preconditioner": (C.c_int, [_P, _P]),
    "gbdmrg_precondition": (C.c_int, [_P, _P, C.c_double, _P, _I32]),
    "gbdmrg_make_pairs": (C.c_int, [_P, _P, _P, C.c_double, _P, C.c_int64, C.c_uint64, _I32, _P, _P, _P, _P,
                                    _PI64]),
    "gbdmrg_set_harvest": (C.c_int, [_P, C.c_int64, _I32, C.c_uint64]),
    "gbdmrg_get_harvest": (C.c_int, [_P, _P, _P, _P, _PI64]),
    "gbdmrg_precond_counters": (C.c_int, [_P, _PI64, _PI64]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1605_02611_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class GbdmrgError(RuntimeError):
    """A library call returned a non-zero status; ``status`` is its name (e.g. "ECUDA")."""

    def __init__(self, msg: str, status: str | None = None):
        super().__init__(msg)
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def mpo_build_host(h1, eri, N: int, two_sz: int = 0, dense: bool = False):
    """Host-only MPO build (no GPU): returns (bond dims, dense matrix or None)."""
    lib = load()
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    K = h1.shape[0]
    prob = Problem(K, N, two_sz, _dptr(h1), _dptr(eri), 0.0)
    dims = np.zeros(K + 1, dtype=np.int32)
    out = np.zeros((4 ** K, 4 ** K)) if dense else None
    st = lib.gbdmrg_mpo_build_host(C.byref(prob), dims.ctypes.data_as(_PI32), _dptr(out) if dense else None)
    if st != 0:
        raise GbdmrgError(f"gbdmrg_mpo_build_host failed: {STATUS.get(st, st)}")
    return dims, out


def kernel_launches() -> int:
    """CUDA kernel launches issued by the library so far in this process."""
    return int(load().gbdmrg_kernel_launches())


def gemm_bf16_selftest(tasks: np.ndarray, terms: np.ndarray, stream: int = 0) -> None:
    """Run the tensor-core grouped GEMM on device buffers (see include/gbdmrg.h)."""
    lib = load()
    tasks = np.ascontiguousarray(tasks, dtype=np.int64)
    terms = np.ascontiguousarray(terms, dtype=np.int64)
    st = lib.gbdmrg_gemm_bf16_selftest(tasks.ctypes.data_as(_PI64), len(tasks), terms.ctypes.data_as(_PI64),
                                       len(terms), _P(stream))
    if st != 0:
        raise GbdmrgError(f"gbdmrg_gemm_bf16_selftest failed: {STATUS.get(st, st)}")


def sigma_flops_host(h1, eri, N: int, two_sz: int, k: int, lab_l, lab_r) -> float:
    """Algorithmic flops of one sigma at sites (k, k+1) (host only, no GPU)."""
    lib = load()
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    prob = Problem(h1.shape[0], N, two_sz, _dptr(h1), _dptr(eri), 0.0)
    ql = np.ascontiguousarray(lab_l, dtype=np.int32).reshape(-1)
    qr = np.ascontiguousarray(lab_r, dtype=np.int32).reshape(-1)
    fl = C.c_double()
    st = lib.gbdmrg_sigma_flops_host(C.byref(prob), k, len(ql) // 2, ql.ctypes.data_as(_PI32), len(qr) // 2,
                                     qr.ctypes.data_as(_PI32), C.byref(fl))
    if st != 0:
        raise GbdmrgError(f"gbdmrg_sigma_flops_host failed: {STATUS.get(st, st)}")
    return fl.value


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class Mlp:
    """Learned Davidson preconditioner network (gbdmrg_mlp_*)."""

    def __init__(self, seed: int = 0, stream: int | None = None):
        self.lib = load()
        self.nparams = int(self.lib.gbdmrg_mlp_nparams())
        h = _P()
        st = self.lib.gbdmrg_mlp_create(seed, _P(stream or 0), C.byref(h))
        if st != 0:
            raise GbdmrgError(f"gbdmrg_mlp_create failed: {STATUS.get(st, st)}")
        self.h = h

    def _check(self, st: int, what: str):
        if st != 0:
            msg = self.lib.gbdmrg_mlp_last_error(self.h).decode()
            raise GbdmrgError(f"{what}: {STATUS.get(st, st)}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.gbdmrg_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.nparams, dtype=np.float32)
        self._check(self.lib.gbdmrg_mlp_get_params(self.h, p.ctypes.data_as(_PF)), "get_params")
        return p

    def set_params(self, p):
        p = _f32(p)
        assert p.size == self.nparams
        self._check(self.lib.gbdmrg_mlp_set_params(self.h, p.ctypes.data_as(_PF)), "set_params")

    def forward(self, F, inference: bool = False) -> np.ndarray:
        F = _f32(F).reshape(-1, 5)
        g = np.zeros(F.shape[0], dtype=np.float32)
        self._check(self.lib.gbdmrg_mlp_forward(self.h, F.ctypes.data_as(_P), F.shape[0], g.ctypes.data_as(_P),
                                                int(inference), 0), "forward")
        return g

    def loss_grad(self, F, P, T):
        F, P, T = _f32(F).reshape(-1, 5), _f32(P), _f32(T)
        g = np.zeros(self.nparams, dtype=np.float32)
        L = C.c_double()
        self._check(self.lib.gbdmrg_mlp_loss_grad(self.h, F.ctypes.data_as(_P), P.ctypes.data_as(_P),
                                                  T.ctypes.data_as(_P), F.shape[0], 0, g.ctypes.data_as(_PF),
                                                  C.byref(L)), "loss_grad")
        return L.value, g

    def train(self, F, P, T, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
        F, P, T = _f32(F).reshape(-1, 5), _f32(P), _f32(T)
        a, b = C.c_double(), C.c_double()
        self._check(self.lib.gbdmrg_mlp_train(self.h, F.ctypes.data_as(_P), P.ctypes.data_as(_P),
                                              T.ctypes.data_as(_P), F.shape[0], 0, epochs, batch, lr, seed,
                                              C.byref(a), C.byref(b)), "train")
        return a.value, b.value


class Batch:
    """Batched tensor-core sigma over several prepared contexts (gbdmrg_batch_*)."""

    def __init__(self, contexts):
        self.lib = load()
        self.ctxs = list(contexts)
        arr = (_P * len(self.ctxs))(*[c.h for c in self.ctxs])
        h = _P()
        st = self.lib.gbdmrg_batch_create(len(self.ctxs), arr, C.byref(h))
        if st != 0:
            msg = self.lib.gbdmrg_last_error(self.ctxs[0].h).decode() if self.ctxs else ""
            raise GbdmrgError(f"gbdmrg_batch_create failed: {STATUS.get(st, st)}: {msg}")
        self.h = h

    def sigma(self, psi_ptrs, sigma_ptrs, use_graph: bool = True):
        """sigma_p = H_eff,p psi_p on device buffers; returns (device ms, algorithmic flops)."""
        n = len(self.ctxs)
        pin = (_P * n)(*psi_ptrs)
        pout = (_P * n)(*sigma_ptrs)
        ms, fl = C.c_double(), C.c_double()
        st = self.lib.gbdmrg_batch_sigma(self.h, pin, pout, int(use_graph), C.byref(ms), C.byref(fl))
        if st != 0:
            msg = self.lib.gbdmrg_batch_last_error(self.h).decode()
            raise GbdmrgError(f"gbdmrg_batch_sigma failed: {STATUS.get(st, st)}: {msg}")
        return ms.value, fl.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.gbdmrg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(contexts, reps: int = 3, splits=None, budgets_mb=None):
    """gbdmrg_autotune over prepared contexts (one: its own sigma; several: the
    batched launch).  Returns (ms per call [nsplits, nbudgets], best split, best budget)."""
    lib = load()
    ctxs = list(contexts)
    arr = (_P * len(ctxs))(*[c.h for c in ctxs])
    sp = None if splits is None else np.ascontiguousarray(splits, dtype=np.float64)
    bu = None if budgets_mb is None else np.ascontiguousarray(budgets_mb, dtype=np.int32)
    ns = 7 if sp is None else len(sp)
    nb = 1 if bu is None else len(bu)
    ms = np.zeros((ns, nb))
    bs, bb = C.c_double(), C.c_int32()
    st = lib.gbdmrg_autotune(len(ctxs), arr, reps, None if sp is None else _dptr(sp), 0 if sp is None else ns,
                             None if bu is None else bu.ctypes.data_as(_PI32), 0 if bu is None else nb,
                             _dptr(ms), C.byref(bs), C.byref(bb))
    if st != 0:
        msg = lib.gbdmrg_last_error(ctxs[0].h).decode() if ctxs else ""
        raise GbdmrgError(f"gbdmrg_autotune failed: {STATUS.get(st, st)}: {msg}")
    return ms, bs.value, bb.value


class Context:
    """One DMRG problem on the current CUDA device (gbdmrg_create)."""

    def __init__(self, h1, eri, N: int, two_sz: int = 0, ecore: float = 0.0, stream: int | None = None):
        self.lib = load()
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        eri = np.ascontiguousarray(eri, dtype=np.float64)
        self.K = h1.shape[0]
        self.N, self.two_sz = N, two_sz
        self.Na, self.Nb = (N + two_sz) // 2, (N - two_sz) // 2
        prob = Problem(self.K, N, two_sz, _dptr(h1), _dptr(eri), ecore)
        h = _P()
        st = self.lib.gbdmrg_create(C.byref(prob), _P(stream or 0), C.byref(h))
        if st != 0:
            raise GbdmrgError(f"gbdmrg_create failed: {STATUS.get(st, st)}")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gbdmrg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != 0:
            msg = self.lib.gbdmrg_last_error(self.h).decode()
            raise GbdmrgError(f"{what}: {STATUS.get(st, st)}: {msg}", STATUS.get(st, str(st)))

    # ---- MPO
    def mpo_bond_dims(self) -> np.ndarray:
        d = np.zeros(self.K + 1, dtype=np.int32)
        self._check(self.lib.gbdmrg_mpo_bond_dims(self.h, d.ctypes.data_as(_PI32)), "mpo_bond_dims")
        return d

    def mpo_dense(self) -> np.ndarray:
        out = np.zeros((4 ** self.K, 4 ** self.K))
        self._check(self.lib.gbdmrg_mpo_dense(self.h, _dptr(out)), "mpo_dense")
        return out

    # ---- MPS
    def set_mps(self, tensors, labels):
        for k, A in enumerate(tensors):
            A = np.ascontiguousarray(A, dtype=np.float64)
            ql = np.ascontiguousarray(labels[k], dtype=np.int32).reshape(-1)
            qr = np.ascontiguousarray(labels[k + 1], dtype=np.int32).reshape(-1)
            self._check(self.lib.gbdmrg_set_mps(self.h, k, A.shape[0], A.shape[2], ql.ctypes.data_as(_PI32),
                                                qr.ctypes.data_as(_PI32), _dptr(A)), f"set_mps({k})")

    def get_mps(self, k: int) -> np.ndarray:
        dl, dr = C.c_int32(), C.c_int32()
        self._check(self.lib.gbdmrg_get_mps(self.h, k, C.byref(dl), C.byref(dr), None), "get_mps")
        A = np.zeros((dl.value, 4, dr.value))
        self._check(self.lib.gbdmrg_get_mps(self.h, k, C.byref(dl), C.byref(dr), _dptr(A)), "get_mps")
        return A

    def get_bond(self, b: int) -> np.ndarray:
        d = C.c_int32()
        self._check(self.lib.gbdmrg_get_bond(self.h, b, C.byref(d), None), "get_bond")
        q = np.zeros((d.value, 2), dtype=np.int32)
        self._check(self.lib.gbdmrg_get_bond(self.h, b, C.byref(d), q.ctypes.data_as(_PI32)), "get_bond")
        return q

    # ---- two-site problem
    def keep_host_plans(self, keep: bool = True):
        self._check(self.lib.gbdmrg_keep_host_plans(self.h, int(keep)), "keep_host_plans")

    def set_chunk_budget(self, megabytes: int):
        """Device memory for the per-chunk sigma intermediates (next prepare)."""
        self._check(self.lib.gbdmrg_set_chunk_budget(self.h, megabytes), "set_chunk_budget")

    def set_split(self, tiles_per_sm: float):
        """Split-K granularity of later tensor-core work lists (tiles per SM; <= 0: none)."""
        self._check(self.lib.gbdmrg_set_split(self.h, float(tiles_per_sm)), "set_split")

    def set_stage1_stacked(self, stacked: bool = True):
        """Stage 1 of later tensor-core work lists over stacked right operands."""
        self._check(self.lib.gbdmrg_set_stage1_stacked(self.h, int(stacked)), "set_stage1_stacked")

    def set_tma_budget(self, megabytes: int):
        """Device memory (MB) for the X intermediates of one precision 4-6 H_eff.psi chunk."""
        self._check(self.lib.gbdmrg_set_tma_budget(self.h, int(megabytes)), "set_tma_budget")

    def set_env_precision(self, precision: int):
        """Environment updates: 0 FP64 units, 2 tensor cores with three BF16 slices,
        3 tensor cores with exactly split operands (FP64-level)."""
        self._check(self.lib.gbdmrg_set_env_precision(self.h, int(precision)), "set_env_precision")

    def set_refinement(self, precision: int, max_iters: int = 8):
        """Second Davidson solve of each tensor-core step with the operator of `precision` (-1: off)."""
        self._check(self.lib.gbdmrg_set_refinement(self.h, int(precision), int(max_iters)), "set_refinement")

    def plan_stats(self) -> dict:
        """Work-list statistics of the prepared precision 4-6 H_eff.psi (see gbdmrg_plan_stats)."""
        out = np.zeros(9)
        self._check(self.lib.gbdmrg_plan_stats(self.h, _dptr(out)), "plan_stats")
        keys = ["stage1_tiles", "stage1_ksteps", "stage2_tiles", "stage2_ksteps", "stage1_exec_flops",
                "stage2_exec_flops", "x_bytes", "rstack_bytes", "chunks"]
        return dict(zip(keys, out.tolist()))

    def set_tc_combos(self, on: bool = True, min_terms: int = 100000):
        """W-contracted sums that feed only the tensor-core sigma and the diagonal on the tensor cores."""
        self._check(self.lib.gbdmrg_set_tc_combos(self.h, int(on), int(min_terms)), "set_tc_combos")

    def plan_params(self):
        """(split tiles per SM, chunk budget MB) of the work lists built next."""
        t, b = C.c_double(), C.c_int32()
        self._check(self.lib.gbdmrg_get_plan_params(self.h, C.byref(t), C.byref(b)), "get_plan_params")
        return t.value, b.value

    def set_precision(self, mode: int):
        """0 FP64, 1 tensor-core BF16 single pass, 2 BF16 x3 slices, 3 BF16 x2 slices;
        4, 5, 6: single pass, three and two slices on the TMA-staged work lists."""
        self._check(self.lib.gbdmrg_set_precision(self.h, mode), "set_precision")

    def prepare(self, k: int):
        self._check(self.lib.gbdmrg_prepare(self.h, k), "prepare")
        nb, nnz = C.c_int64(), C.c_int64()
        self._check(self.lib.gbdmrg_psi_layout(self.h, C.byref(nb), C.byref(nnz), None), "psi_layout")
        blk = np.zeros((nb.value, 7), dtype=np.int64)
        self._check(self.lib.gbdmrg_psi_layout(self.h, C.byref(nb), C.byref(nnz), blk.ctypes.data_as(_PI64)),
                    "psi_layout")
        self.layout = blk
        self.nnz = nnz.value
        return blk

    def plan(self, k: int):
        """Rebuild the H_eff work lists at (k, k+1) from the held environments."""
        self._check(self.lib.gbdmrg_plan(self.h, k), "plan")

    def pack(self, psi: np.ndarray) -> np.ndarray:
        out = np.zeros(self.nnz)
        for (l0, ld, n1, n2, r0, rd, off) in self.layout:
            out[off:off + ld * rd] = psi[l0:l0 + ld, n1, n2, r0:r0 + rd].reshape(-1)
        return out

    def unpack(self, v: np.ndarray, shape) -> np.ndarray:
        out = np.zeros(shape)
        for (l0, ld, n1, n2, r0, rd, off) in self.layout:
            out[l0:l0 + ld, n1, n2, r0:r0 + rd] = v[off:off + ld * rd].reshape(ld, rd)
        return out

    def sigma(self, psi_packed: np.ndarray):
        x = np.ascontiguousarray(psi_packed, dtype=np.float64)
        y = np.zeros_like(x)
        fl = C.c_double()
        self._check(self.lib.gbdmrg_sigma(self.h, x.ctypes.data_as(_P), y.ctypes.data_as(_P), 0, C.byref(fl)),
                    "sigma")
        return y, fl.value

    def sigma_device(self, x_ptr: int, y_ptr: int) -> float:
        fl = C.c_double()
        self._check(self.lib.gbdmrg_sigma(self.h, _P(x_ptr), _P(y_ptr), 1, C.byref(fl)), "sigma")
        return fl.value

    def sigma_timing(self, reps: int, x_ptr: int, y_ptr: int) -> float:
        ms = C.c_double()
        self._check(self.lib.gbdmrg_sigma_timing(self.h, reps, _P(x_ptr), _P(y_ptr), C.byref(ms)), "sigma_timing")
        return ms.value

    def diag(self) -> np.ndarray:
        d = np.zeros(self.nnz)
        self._check(self.lib.gbdmrg_diag(self.h, d.ctypes.data_as(_P), 0), "diag")
        return d

    def step(self, k: int, direction: int, M: int, tol: float, max_iter: int, psi_in=None, want_psi=False,
             on_device: bool = False):
        """One two-site update (gbdmrg_step).  Host numpy (or device pointers if on_device)."""
        e, d, it = C.c_double(), C.c_double(), C.c_int32()
        pin = pout = None
        out = None
        if on_device:
            pin = _P(psi_in) if psi_in is not None else None
            pout = _P(want_psi) if want_psi else None
        else:
            if psi_in is not None:
                psi_in = np.ascontiguousarray(psi_in, dtype=np.float64)
                pin = psi_in.ctypes.data_as(_P)
            if want_psi:
                out = np.zeros(self.nnz)
                pout = out.ctypes.data_as(_P)
        self._check(self.lib.gbdmrg_step(self.h, k, direction, M, tol, max_iter, pin, pout, int(on_device),
                                         C.byref(e), C.byref(d), C.byref(it)), "step")
        return e.value, d.value, it.value, out

    def phase_times(self):
        t = np.zeros(8)
        self._check(self.lib.gbdmrg_phase_times(self.h, _dptr(t)), "phase_times")
        return dict(zip(["tilde", "plan", "diag", "davidson", "decimate", "env_update"], t[:6].tolist()))

    def phase_flops(self):
        t = np.zeros(8)
        self._check(self.lib.gbdmrg_phase_flops(self.h, _dptr(t)), "phase_flops")
        return dict(zip(["tilde", "plan", "diag", "davidson", "decimate", "env_update"], t[:6].tolist()))

    def counters(self):
        f, s, o = C.c_double(), C.c_double(), C.c_double()
        n = C.c_int64()
        self._check(self.lib.gbdmrg_counters(self.h, C.byref(f), C.byref(s), C.byref(n), C.byref(o)), "counters")
        return dict(sigma_flops=f.value, sigma_seconds=s.value, sigma_calls=n.value, other_flops=o.value)

    def expectation(self) -> float:
        """<psi|H|psi>/<psi|psi> + ecore of the current MPS at the prepared position."""
        v = C.c_double()
        self._check(self.lib.gbdmrg_expectation(self.h, C.byref(v)), "expectation")
        return v.value

    # ---- checkpoint
    def save(self, path: str):
        """Write the MPS to a checkpoint file (gbdmrg_save)."""
        self._check(self.lib.gbdmrg_save(self.h, os.fsencode(path)), "save")

    def load(self, path: str):
        """Replace the MPS by the one in a checkpoint file (gbdmrg_load)."""
        self._check(self.lib.gbdmrg_load(self.h, os.fsencode(path)), "load")

    # ---- learned preconditioner
    def set_preconditioner(self, mlp):
        """Use the network `mlp` (an Mlp) in Davidson, or the diagonal one when None."""
        self._mlp = mlp
        self._check(self.lib.gbdmrg_set_preconditioner(self.h, mlp.h if mlp is not None else None),
                    "set_preconditioner")

    def precondition(self, r, theta: float) -> np.ndarray:
        r = np.ascontiguousarray(r, dtype=np.float64)
        t = np.zeros_like(r)
        self._check(self.lib.gbdmrg_precondition(self.h, r.ctypes.data_as(_P), theta, t.ctypes.data_as(_P), 0),
                    "precondition")
        return t

    def make_pairs(self, x, r, theta: float, psi, ns: int, seed: int):
        x, r, psi = (np.ascontiguousarray(v, dtype=np.float64) for v in (x, r, psi))
        F = np.zeros((ns, 5), dtype=np.float32)
        P = np.zeros(ns, dtype=np.float32)
        T = np.zeros(ns, dtype=np.float32)
        idx = np.zeros(ns, dtype=np.int64)
        w = C.c_int64()
        self._check(self.lib.gbdmrg_make_pairs(self.h, x.ctypes.data_as(_P), r.ctypes.data_as(_P), theta,
                                               psi.ctypes.data_as(_P), ns, seed, 0, F.ctypes.data_as(_P),
                                               P.ctypes.data_as(_P), T.ctypes.data_as(_P), idx.ctypes.data_as(_P),
                                               C.byref(w)), "make_pairs")
        k = w.value
        return F[:k], P[:k], T[:k], idx[:k]

    def set_harvest(self, capacity: int, per_iteration: int, seed: int = 0):
        self._check(self.lib.gbdmrg_set_harvest(self.h, capacity, per_iteration, seed), "set_harvest")

    def get_harvest(self):
        n = C.c_int64()
        self._check(self.lib.gbdmrg_get_harvest(self.h, None, None, None, C.byref(n)), "get_harvest")
        F = np.zeros((n.value, 5), dtype=np.float32)
        P = np.zeros(n.value, dtype=np.float32)
        T = np.zeros(n.value, dtype=np.float32)
        if n.value:
            self._check(self.lib.gbdmrg_get_harvest(self.h, F.ctypes.data_as(_P), P.ctypes.data_as(_P),
                                                    T.ctypes.data_as(_P), C.byref(n)), "get_harvest")
        return F, P, T

    def precond_counters(self):
        a, b = C.c_int64(), C.c_int64()
        self._check(self.lib.gbdmrg_precond_counters(self.h, C.byref(a), C.byref(b)), "precond_counters")
        return dict(learned=a.value, fallbacks=b.value)

    def diag_noalloc(self, diag_ptr: int):
        """Diagonal of H_eff into a device buffer without device allocation."""
        self._check(self.lib.gbdmrg_diag_noalloc(self.h, _P(diag_ptr)), "diag_noalloc")

    # ---- sweeps
    def run(self, M, dav_tol, max_iter: int = 200, precision: int = 0):
        M = np.ascontiguousarray(M, dtype=np.int32)
        tol = np.ascontiguousarray(np.broadcast_to(dav_tol, M.shape), dtype=np.float64)
        s = Schedule(len(M), M.ctypes.data_as(_PI32), _dptr(tol), max_iter, precision)
        e = np.zeros(len(M))
        d = np.zeros(len(M))
        self._check(self.lib.gbdmrg_run(self.h, C.byref(s), _dptr(e), _dptr(d)), "run")
        sec, fl, ss = np.zeros(len(M)), np.zeros(len(M)), np.zeros(len(M))
        it = np.zeros(len(M), dtype=np.int32)
        self._check(self.lib.gbdmrg_run_stats(self.h, _dptr(sec), _dptr(fl), _dptr(ss), it.ctypes.data_as(_PI32)),
                    "run_stats")
        return dict(energy=e, discarded=d, seconds=sec, sigma_flops=fl, sigma_seconds=ss, davidson_iters=it)
