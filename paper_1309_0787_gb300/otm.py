"""Python binding of the C ABI in ``include/otm.h`` (argument marshalling only).

Every function takes and returns PyTorch CUDA tensors and forwards to the
entry point of the same name in ``_build/libotm.so`` on the current CUDA
stream.  All arithmetic runs in the library's CUDA kernels; there is no
fallback: if the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libotm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libotm.so not built ({LIB_PATH}); run python -m paper_1309_0787_gb300.build")

_lib = ctypes.CDLL(LIB_PATH)

c_i64 = ctypes.c_int64
c_f64 = ctypes.c_double
c_vp = ctypes.c_void_p
c_sz = ctypes.c_size_t


class OtmCsr(ctypes.Structure):
    _fields_ = [("rows", c_i64), ("cols", c_i64), ("nnz", c_i64), ("row_ptr", c_vp),
                ("col", c_vp), ("val", c_vp)]


_P = ctypes.POINTER(OtmCsr)


class OtmProblem(ctypes.Structure):
    _fields_ = [("n", c_i64), ("k", c_i64), ("b", c_i64), ("epochs", c_i64), ("Yq", c_vp),
                ("scales", c_vp), ("perm", c_vp), ("ybar3", c_vp), ("V", c_vp),
                ("restarts", c_i64), ("beta0", c_f64), ("theta", c_f64), ("alpha0", c_f64)]


class OtmBatchPlan(ctypes.Structure):
    _fields_ = [("nitems", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_k", ctypes.c_int32),
                ("grid_clusters", ctypes.c_int32), ("nitems_wide", ctypes.c_int32),
                ("grid_clusters_wide", ctypes.c_int32), ("max_k_wide", ctypes.c_int32),
                ("cluster_wide", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("vimg2", ctypes.c_int32), ("stages_wide", ctypes.c_int32),
                ("vimg2_wide", ctypes.c_int32), ("smem_bytes", c_i64), ("ws", c_vp),
                ("ws_bytes", c_sz)]


class OtmMlp(ctypes.Structure):
    _fields_ = [("d_in", c_i64), ("width", c_i64), ("d_out", c_i64), ("p", c_vp), ("p16", c_vp),
                ("w2t16", c_vp), ("w3t16", c_vp), ("grad", c_vp), ("adam_m", c_vp),
                ("adam_v", c_vp)]


_MP = ctypes.POINTER(OtmMlp)
_PP = ctypes.POINTER(OtmProblem)
_BP = ctypes.POINTER(OtmBatchPlan)

# entry point -> argument types (every entry returns int status unless listed below)
_SIGS = {
    "otm_version": [],
    "otm_last_error": [],
    "otm_launch_count": [],
    "otm_topic_moments": [_P, c_vp, c_vp, c_vp, c_vp, c_vp],
    "otm_topic_m2_workspace": [c_i64, c_i64],
    "otm_topic_m2_apply": [_P, _P, c_vp, c_vp, c_vp, c_f64, c_vp, c_i64, c_vp, c_vp, c_sz,
                           c_vp],
    "otm_csr_transpose_workspace": [c_i64, c_i64],
    "otm_csr_transpose": [_P, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp],
    "otm_pairs_workspace": [c_i64, c_i64],
    "otm_pairs_apply": [_P, _P, c_vp, c_i64, c_vp, c_vp, c_sz, c_vp],
    "otm_orth_workspace": [c_i64],
    "otm_orthonormalize": [c_vp, c_i64, c_i64, c_vp, c_sz, c_vp],
    "otm_syev_workspace": [c_i64],
    "otm_syev": [c_vp, c_i64, c_vp, c_vp, c_vp, c_sz, c_vp],
    "otm_syev_noalloc": [c_vp, c_i64, c_vp, c_vp, c_vp],
    "otm_whiten_topic_workspace": [c_i64, c_i64, c_i64, c_i64, c_i64],
    "otm_whiten_topic": [_P, c_vp, c_i64, c_i64, ctypes.c_int, c_f64, c_vp, c_vp, c_vp, c_vp,
                         c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp],
    "otm_whiten_topic_nystrom_workspace": [c_i64, c_i64, c_i64, c_i64],
    "otm_whiten_topic_nystrom": [_P, c_vp, c_i64, c_i64, c_f64, c_vp, c_vp, c_vp, c_vp, c_vp,
                                 c_vp, c_vp, c_vp, c_vp, c_sz, c_vp],
    "otm_whiten_community_workspace": [c_i64, c_i64, c_i64, c_i64, c_i64, c_i64],
    "otm_whiten_community": [_P, _P, _P, c_vp, c_vp, c_i64, c_i64, ctypes.c_int, c_f64, c_vp,
                             c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp],
    "otm_project": [_P, c_vp, c_i64, c_vp, c_vp, c_vp],
    "otm_column_mean": [c_vp, c_i64, c_i64, c_vp, c_vp],
    "otm_sgd_step": [c_vp, c_vp, c_vp, c_vp, c_i64, c_i64, c_vp, c_f64, c_f64, c_f64, c_vp, c_sz,
                     c_vp],
    "otm_sgd_workspace": [c_i64, c_i64],
    "otm_sgd_set_form": [ctypes.c_int],
    "otm_sgd_split_shape": [c_i64, c_i64, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int)],
    "otm_sgd_run": [c_vp, c_vp, c_vp, c_vp, c_i64, c_i64, c_vp, c_vp, c_i64, c_i64, c_f64,
                    c_f64, c_f64, c_i64, c_vp, c_vp, c_sz, c_vp],
    "otm_sgd_topic_exact_workspace": [c_i64, c_i64, c_i64, ctypes.c_int],
    "otm_sgd_run_topic_exact": [c_vp, _P, c_vp, c_vp, c_i64, c_vp, c_i64, c_i64, c_i64, c_f64,
                                c_f64, c_f64, ctypes.c_int, c_vp, c_i64, c_vp, c_sz, c_vp],
    "otm_quantize_samples": [c_vp, c_i64, c_i64, ctypes.c_int, c_vp, c_vp, c_vp],
    "otm_sgd_run_lp_workspace": [],
    "otm_sgd_run_lp": [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, c_i64, c_vp, c_vp, c_i64,
                       c_i64, c_f64, c_f64, c_f64, ctypes.c_int, c_i64, c_vp, c_vp, c_sz, c_vp],
    "otm_sgd_batched_workspace": [c_i64],
    "otm_sgd_batched_prepare": [_PP, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_vp, c_sz, _BP,
                                c_vp],
    "otm_sgd_batched_launch": [_BP, c_vp],
    "otm_sgd_batched_check": [_BP, c_vp],
    "otm_mlp_param_count": [c_i64, c_i64, c_i64],
    "otm_mlp_sync_weights": [_MP, c_vp],
    "otm_mlp_workspace": [_MP, c_i64],
    "otm_mlp_forward": [_MP, c_vp, c_i64, c_vp, c_vp, c_sz, c_vp],
    "otm_mlp_backward": [_MP, c_vp, c_i64, c_vp, c_vp, c_sz, c_vp],
    "otm_adam_step": [_MP, c_f64, c_f64, c_f64, c_f64, c_i64, c_vp],
    "otm_gram_schmidt": [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp],
    "otm_gram_schmidt_backward": [c_vp, c_vp, c_vp, c_i64, c_i64, c_vp, c_vp],
    "otm_ws_loss_grad": [c_vp, c_vp, c_vp, c_i64, c_i64, c_f64, c_vp, c_vp, c_vp],
    "otm_ws_train_workspace": [_MP, c_i64],
    "otm_ws_train_step": [_MP, c_vp, c_vp, c_vp, c_i64, c_i64, c_f64, c_i64, c_vp, c_vp, c_sz,
                          c_vp],
    "otm_ws_infer": [_MP, c_vp, c_i64, c_i64, c_vp, c_vp, c_sz, c_vp],
    "otm_ws_check": [c_vp, c_vp],
    "otm_ws_canonicalize": [c_vp, c_i64, c_i64, ctypes.c_int, c_vp, c_vp, c_vp, c_vp],
    "otm_ws_rotate": [c_vp, c_vp, c_i64, c_i64, ctypes.c_int, c_vp, c_vp],
    "otm_ws_sketch_workspace": [c_i64, c_i64, c_i64, ctypes.c_int],
    "otm_ws_sketch": [c_vp, c_i64, c_i64, c_i64, c_vp, c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_sz,
                      c_vp],
    "otm_ws_init_workspace": [c_i64, c_i64, c_i64],
    "otm_ws_init_components": [c_vp, c_vp, c_i64, c_i64, c_i64, c_vp, c_f64, c_vp, c_vp, c_sz,
                               c_vp],
    "otm_ws_generate": [c_vp, c_vp, c_i64, c_i64, c_i64, ctypes.c_uint64, c_i64, c_vp, c_vp],
    "otm_gemm_bf16_workspace": [],
    "otm_gemm_bf16": [c_vp, c_vp, c_i64, c_i64, c_i64, c_i64, c_i64, c_i64, c_i64, c_i64,
                      ctypes.c_int, ctypes.c_float, c_vp, c_vp, c_i64, c_i64, c_vp, c_i64, c_i64,
                      c_vp, c_sz, c_vp],
    "otm_unwhiten_workspace": [c_i64, c_i64, c_i64],
    "otm_unwhiten": [c_vp, c_i64, c_vp, c_i64, c_i64, c_vp, c_f64, ctypes.c_int, c_vp, c_vp,
                     c_vp, c_vp, c_sz, c_vp],
    "otm_recon_error_workspace": [c_i64],
    "otm_recon_error": [c_vp, c_i64, c_f64, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp],
    "otm_membership_workspace": [c_i64],
    "otm_membership": [c_vp, c_i64, c_i64, c_vp, c_f64, c_f64, c_vp, c_vp, c_sz, c_vp],
    "otm_pvalue_match_workspace": [c_i64, c_i64],
    "otm_pvalue_match": [c_vp, c_i64, c_vp, c_i64, c_i64, c_f64, c_vp, c_vp, c_vp, c_vp, c_sz,
                         c_vp],
}
_RESTYPE = {"otm_last_error": ctypes.c_char_p, "otm_version": ctypes.c_int,
            "otm_launch_count": ctypes.c_uint64, "otm_mlp_param_count": c_i64}

for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _RESTYPE.get(_name, c_sz if _name.endswith("_workspace") else ctypes.c_int)

STATUS = {0: "OTM_OK", 1: "OTM_EINVAL", 2: "OTM_ENOTPSD", 3: "OTM_ENOMEM", 4: "OTM_ECUDA",
          5: "OTM_ETIMEOUT", 6: "OTM_ENOTCONVERGED"}


class OtmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def _check(st: int) -> None:
    if st != 0:
        raise OtmError(st, _lib.otm_last_error().decode())


def version() -> int:
    return _lib.otm_version()


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(_lib.otm_launch_count())


def _stream():
    return c_vp(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    # the library launches on the current device and stream: a tensor that lives
    # on another GPU would be dereferenced by a kernel on this one
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"tensor on {t.device}, but the current CUDA device is "
                         f"cuda:{torch.cuda.current_device()}")
    return c_vp(t.data_ptr())


def _need(t, dtype, shape, name):
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")


def _ws(nbytes: int, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


class DeviceCSR:
    """CSR matrix resident on the GPU (int32 row_ptr/col, float32 values)."""

    def __init__(self, row_ptr, col, val, shape):
        self.row_ptr, self.col, self.val = row_ptr, col, val
        self.shape = (int(shape[0]), int(shape[1]))
        self._desc = OtmCsr(self.shape[0], self.shape[1], int(col.numel()),
                            row_ptr.data_ptr(), col.data_ptr() if col.numel() else 0,
                            val.data_ptr() if val.numel() else 0)

    @classmethod
    def from_host(cls, csr, device="cuda"):
        rp = torch.as_tensor(csr.row_ptr, dtype=torch.int32).to(device)
        col = torch.as_tensor(csr.col, dtype=torch.int32).to(device)
        val = torch.as_tensor(csr.val, dtype=torch.float32).to(device)
        return cls(rp, col, val, csr.shape)

    @property
    def nnz(self):
        return int(self.col.numel())

    @property
    def device(self):
        return self.row_ptr.device

    def ref(self):
        if not self.row_ptr.is_cuda or self.row_ptr.device.index != torch.cuda.current_device():
            raise ValueError(f"CSR on {self.row_ptr.device}, but the current CUDA device is "
                             f"cuda:{torch.cuda.current_device()}")
        return ctypes.byref(self._desc)


# --------------------------------------------------------------------------
def topic_moments(X: DeviceCSR) -> dict:
    n, d = X.shape
    dev = X.device
    out = {"row_invlen": torch.empty(n, dtype=torch.float32, device=dev),
           "row_w": torch.empty(n, dtype=torch.float32, device=dev),
           "M1": torch.empty(d, dtype=torch.float64, device=dev),
           "delta": torch.empty(d, dtype=torch.float64, device=dev)}
    _check(_lib.otm_topic_moments(X.ref(), _ptr(out["row_invlen"]), _ptr(out["row_w"]),
                                  _ptr(out["M1"]), _ptr(out["delta"]), _stream()))
    return out


def csr_transpose(X: DeviceCSR) -> DeviceCSR:
    """The CSR of X^T (d x n); within a word the documents come in no fixed order."""
    n, d = X.shape
    dev = X.device
    colptr = torch.empty(d + 1, dtype=torch.int32, device=dev)
    rowT = torch.empty(X.nnz, dtype=torch.int32, device=dev)
    valT = torch.empty(X.nnz, dtype=torch.float32, device=dev)
    ws = _ws(_lib.otm_csr_transpose_workspace(n, d), dev)
    _check(_lib.otm_csr_transpose(X.ref(), _ptr(colptr), _ptr(rowT), _ptr(valT), _ptr(ws),
                                  ws.numel(), _stream()))
    return DeviceCSR(colptr, rowT, valT, (d, n))


def topic_m2_apply(X: DeviceCSR, moments: dict, alpha0: float, S, Xt: DeviceCSR = None):
    n, d = X.shape
    m = S.shape[1]
    _need(S, torch.float32, (d, m), "S")
    O = torch.empty_like(S)
    ws = _ws(_lib.otm_topic_m2_workspace(n, m), S.device)
    _check(_lib.otm_topic_m2_apply(X.ref(), Xt.ref() if Xt is not None else None,
                                   _ptr(moments["row_w"]), _ptr(moments["M1"]),
                                   _ptr(moments["delta"]), float(alpha0), _ptr(S), m, _ptr(O),
                                   _ptr(ws), ws.numel(), _stream()))
    return O


def pairs_apply(G1: DeviceCSR, G2: DeviceCSR, S):
    m = S.shape[1]
    _need(S, torch.float32, (G2.shape[1], m), "S")
    O = torch.empty(G1.shape[1], m, dtype=torch.float32, device=S.device)
    ws = _ws(_lib.otm_pairs_workspace(G1.shape[0], m), S.device)
    _check(_lib.otm_pairs_apply(G1.ref(), G2.ref(), _ptr(S), m, _ptr(O), _ptr(ws), ws.numel(),
                                _stream()))
    return O


def orthonormalize(A):
    rows, m = A.shape
    _need(A, torch.float32, (rows, m), "A")
    ws = _ws(_lib.otm_orth_workspace(m), A.device)
    _check(_lib.otm_orthonormalize(_ptr(A), rows, m, _ptr(ws), ws.numel(), _stream()))
    return A


def syev(A):
    n = A.shape[0]
    _need(A, torch.float64, (n, n), "A")
    ev = torch.empty(n, dtype=torch.float64, device=A.device)
    vec = torch.empty(n, n, dtype=torch.float64, device=A.device)
    ws = _ws(_lib.otm_syev_workspace(n), A.device)
    _check(_lib.otm_syev(_ptr(A), n, _ptr(ev), _ptr(vec), _ptr(ws), ws.numel(), _stream()))
    return ev, vec


def syev_noalloc(A, evals, evecs) -> None:
    """otm_syev_noalloc: the library allocates nothing (scratch is a fixed
    array inside it, n <= 160); the caller provides the outputs evals (n,
    float64) and evecs (n x n, float64)."""
    n = A.shape[0]
    _need(A, torch.float64, (n, n), "A")
    _need(evals, torch.float64, (n,), "evals")
    _need(evecs, torch.float64, (n, n), "evecs")
    _check(_lib.otm_syev_noalloc(_ptr(A), n, _ptr(evals), _ptr(evecs), _stream()))


def whiten_topic(X: DeviceCSR, S, k: int, power_iters: int, alpha0: float) -> dict:
    n, d = X.shape
    kt = S.shape[1]
    _need(S, torch.float32, (d, kt), "S")
    dev = S.device
    f32, f64 = torch.float32, torch.float64
    o = {"W": torch.empty(d, k, dtype=f32, device=dev), "Q": torch.empty(d, kt, dtype=f32, device=dev),
         "Cw": torch.empty(kt, k, dtype=f64, device=dev), "Cp": torch.empty(kt, k, dtype=f64, device=dev),
         "eig": torch.empty(k, dtype=f64, device=dev), "M1": torch.empty(d, dtype=f64, device=dev),
         "row_invlen": torch.empty(n, dtype=f32, device=dev),
         "row_w": torch.empty(n, dtype=f32, device=dev)}
    ws = _ws(_lib.otm_whiten_topic_workspace(n, d, X.nnz, k, kt), dev)
    _check(_lib.otm_whiten_topic(X.ref(), _ptr(S), k, kt, int(power_iters), float(alpha0),
                                 _ptr(o["W"]), _ptr(o["Q"]), _ptr(o["Cw"]), _ptr(o["Cp"]),
                                 _ptr(o["eig"]), _ptr(o["M1"]), _ptr(o["row_invlen"]),
                                 _ptr(o["row_w"]), _ptr(ws), ws.numel(), _stream()))
    return o


def whiten_topic_nystrom(X: DeviceCSR, S, k: int, alpha0: float) -> dict:
    """otm_whiten_topic_nystrom (Algorithm 2); "Q" holds O = M2 S."""
    n, d = X.shape
    kt = S.shape[1]
    _need(S, torch.float32, (d, kt), "S")
    dev = S.device
    f32, f64 = torch.float32, torch.float64
    o = {"W": torch.empty(d, k, dtype=f32, device=dev), "Q": torch.empty(d, kt, dtype=f32, device=dev),
         "Cw": torch.empty(kt, k, dtype=f64, device=dev), "Cp": torch.empty(kt, k, dtype=f64, device=dev),
         "eig": torch.empty(k, dtype=f64, device=dev), "M1": torch.empty(d, dtype=f64, device=dev),
         "row_invlen": torch.empty(n, dtype=f32, device=dev),
         "row_w": torch.empty(n, dtype=f32, device=dev)}
    ws = _ws(_lib.otm_whiten_topic_nystrom_workspace(n, d, k, kt), dev)
    _check(_lib.otm_whiten_topic_nystrom(X.ref(), _ptr(S), k, kt, float(alpha0), _ptr(o["W"]),
                                         _ptr(o["Q"]), _ptr(o["Cw"]), _ptr(o["Cp"]), _ptr(o["eig"]),
                                         _ptr(o["M1"]), _ptr(o["row_invlen"]), _ptr(o["row_w"]),
                                         _ptr(ws), ws.numel(), _stream()))
    return o


def whiten_community(G_XA: DeviceCSR, G_XB: DeviceCSR, G_XC: DeviceCSR, S_pairs, S_w, k: int,
                     power_iters: int, alpha0: float) -> dict:
    nx, na = G_XA.shape
    nb, nc = G_XB.shape[1], G_XC.shape[1]
    kt = S_w.shape[1]
    _need(S_w, torch.float32, (na, kt), "S_w")
    _need(S_pairs, torch.float32, (nb, kt), "S_pairs")
    dev = S_w.device
    f32, f64 = torch.float32, torch.float64
    o = {"W": torch.empty(na, k, dtype=f32, device=dev), "W_B": torch.empty(nb, k, dtype=f32, device=dev),
         "W_C": torch.empty(nc, k, dtype=f32, device=dev), "Q": torch.empty(na, kt, dtype=f32, device=dev),
         "Cw": torch.empty(kt, k, dtype=f64, device=dev), "Cp": torch.empty(kt, k, dtype=f64, device=dev),
         "eig": torch.empty(k, dtype=f64, device=dev), "sigma": torch.empty(k, dtype=f64, device=dev),
         "M1": torch.empty(na, dtype=f64, device=dev)}
    ws = _ws(_lib.otm_whiten_community_workspace(nx, na, nb, nc, k, kt), dev)
    _check(_lib.otm_whiten_community(G_XA.ref(), G_XB.ref(), G_XC.ref(), _ptr(S_pairs), _ptr(S_w),
                                     k, kt, int(power_iters), float(alpha0), _ptr(o["W"]),
                                     _ptr(o["W_B"]), _ptr(o["W_C"]), _ptr(o["Q"]), _ptr(o["Cw"]),
                                     _ptr(o["Cp"]), _ptr(o["eig"]), _ptr(o["sigma"]),
                                     _ptr(o["M1"]), _ptr(ws), ws.numel(), _stream()))
    return o


def project(X: DeviceCSR, W, row_scale=None):
    n, d = X.shape
    k = W.shape[1]
    _need(W, torch.float32, (d, k), "W")
    if row_scale is not None:
        _need(row_scale, torch.float32, (n,), "row_scale")
    Y = torch.empty(n, k, dtype=torch.float32, device=W.device)
    _check(_lib.otm_project(X.ref(), _ptr(W), k, _ptr(row_scale), _ptr(Y), _stream()))
    return Y


def column_mean(Y, out=None):
    """ybar (k, float64); written into `out` (a contiguous float64 k-vector) if given."""
    n, k = Y.shape
    _need(Y, torch.float32, (n, k), "Y")
    yb = torch.empty(k, dtype=torch.float64, device=Y.device) if out is None else out
    _need(yb, torch.float64, (k,), "out")
    _check(_lib.otm_column_mean(_ptr(Y), n, k, _ptr(yb), _stream()))
    return yb


SGD_FORM_AUTO, SGD_FORM_CLUSTER, SGD_FORM_GRID, SGD_FORM_SPLIT = 0, 1, 2, 3


def sgd_set_form(form: int) -> None:
    """otm_sgd_set_form: which FP32 kernel sgd_step / sgd_run use (process-wide)."""
    _check(_lib.otm_sgd_set_form(int(form)))


def sgd_split_shape(k: int, b: int, sym: bool):
    """(clusters, CTAs per cluster) of the split form for k, b and the views, or
    (0, 0) where it does not apply on the current device."""
    c, cl = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib.otm_sgd_split_shape(int(k), int(b), int(bool(sym)), ctypes.byref(c),
                                    ctypes.byref(cl)))
    return c.value, cl.value


def sgd_step(V, YA, YB, YC, ybar3, theta: float, beta: float, alpha0: float):
    k = V.shape[0]
    b = YA.shape[0]
    _need(V, torch.float32, (k, k), "V")
    for nm, Y in (("YA", YA), ("YB", YB), ("YC", YC)):
        _need(Y, torch.float32, (b, k), nm)
    _need(ybar3, torch.float64, (3, k), "ybar3")
    ws = _ws(_lib.otm_sgd_workspace(k, b), V.device)
    _check(_lib.otm_sgd_step(_ptr(V), _ptr(YA), _ptr(YB), _ptr(YC), b, k, _ptr(ybar3),
                             float(theta), float(beta), float(alpha0), _ptr(ws), ws.numel(),
                             _stream()))
    return V


def sgd_run(V, YA, YB, YC, ybar3, perm, epochs: int, b: int, beta0: float, theta: float,
            alpha0: float, snapshot_every: int = 0):
    """V is k x k column-major as stored (V[i] = component i); updated in place.
    Returns the snapshot tensor (steps // snapshot_every, k, k) or None."""
    k = V.shape[0]
    n = YA.shape[0]
    _need(V, torch.float32, (k, k), "V")
    for nm, Y in (("YA", YA), ("YB", YB), ("YC", YC)):
        _need(Y, torch.float32, (n, k), nm)
    _need(ybar3, torch.float64, (3, k), "ybar3")
    if perm is not None:
        _need(perm, torch.int32, (epochs, n), "perm")
    steps = ((n + b - 1) // b) * epochs
    snaps = None
    if snapshot_every:
        snaps = torch.empty(max(steps // snapshot_every, 1), k, k, dtype=torch.float32,
                            device=V.device)
    ws = _ws(_lib.otm_sgd_workspace(k, int(b)), V.device)
    _check(_lib.otm_sgd_run(_ptr(V), _ptr(YA), _ptr(YB), _ptr(YC), n, k, _ptr(ybar3),
                            _ptr(perm), int(epochs), int(b), float(beta0), float(theta),
                            float(alpha0), int(snapshot_every), _ptr(snaps), _ptr(ws), ws.numel(),
                            _stream()))
    return snaps


PREC_BF16 = 1
PREC_FP8 = 2
PREC_FP8X2 = 3  # e4m3, samples and B as two terms (sgd_run_lp only)


def sgd_run_topic_exact(V, X: DeviceCSR, W, M1, perm, epochs: int, b: int, beta0: float,
                        theta: float, alpha0: float, snapshot_every: int = 0,
                        precision: int = 0):
    """otm_sgd_run_topic_exact: STGD on the whole third moment of Eq. (3) (the
    self-token terms kept).  V: k x k (V[i] = component i), W: d x k float32,
    M1: d float64, perm: epochs x n int32 or None; precision 0 (FP32) or
    PREC_BF16 (the two large products on the tensor cores).  The workspace is
    sized by the most word occurrences any minibatch holds (from the row
    pointers)."""
    k = V.shape[0]
    n, d = X.shape
    _need(V, torch.float32, (k, k), "V")
    _need(W, torch.float32, (d, k), "W")
    _need(M1, torch.float64, (d,), "M1")
    if perm is not None:
        _need(perm, torch.int32, (epochs, n), "perm")
    # the workspace holds the largest minibatch's word occurrences (host-side
    # sizing from the row pointers and the visiting order)
    per = np.diff(X.row_ptr.cpu().numpy().astype(np.int64))
    order = (perm.cpu().numpy().astype(np.int64) if perm is not None
             else np.tile(np.arange(n, dtype=np.int64), (max(epochs, 1), 1)))
    starts = np.arange(0, n, b)
    ends = np.minimum(starts + b, n)
    cap = 0
    for e in range(epochs):
        valid = (order[e] >= 0) & (order[e] < n)
        cs = np.concatenate([[0], np.cumsum(np.where(valid, per[np.clip(order[e], 0, n - 1)], 0))])
        cap = max(cap, int((cs[ends] - cs[starts]).max()))
    steps = ((n + b - 1) // b) * epochs
    snaps = None
    if snapshot_every:
        snaps = torch.empty(max(steps // snapshot_every, 1), k, k, dtype=torch.float32,
                            device=V.device)
    ws = _ws(_lib.otm_sgd_topic_exact_workspace(k, min(b, n), cap, int(precision)), V.device)
    _check(_lib.otm_sgd_run_topic_exact(_ptr(V), X.ref(), _ptr(W), _ptr(M1), k, _ptr(perm),
                                        int(epochs), int(b), cap, float(beta0), float(theta),
                                        float(alpha0), int(precision), _ptr(snaps),
                                        int(snapshot_every), _ptr(ws), ws.numel(), _stream()))
    return snaps


def quantize_samples(Y, precision: int):
    """Samples for the tensor-core STGD: returns (Yq, scales), Yq n x ldq
    (ldq = k rounded up to 16) BF16 or FP8 e4m3 stored as bytes (2 n rows for
    PREC_FP8X2: the second e4m3 terms after the first), scales n."""
    n, k = Y.shape
    _need(Y, torch.float32, (n, k), "Y")
    ldq = (k + 15) // 16 * 16
    es = 2 if precision == PREC_BF16 else 1
    rows = 2 * n if precision == PREC_FP8X2 else n
    Yq = torch.empty(rows, ldq * es, dtype=torch.uint8, device=Y.device)
    sc = torch.empty(n, dtype=torch.float32, device=Y.device)
    _check(_lib.otm_quantize_samples(_ptr(Y), n, k, int(precision), _ptr(Yq), _ptr(sc), _stream()))
    return Yq, sc


def sgd_run_lp(V, YA, YB, YC, ybar3, perm, epochs: int, b: int, beta0: float, theta: float,
               alpha0: float, precision: int, snapshot_every: int = 0):
    """Tensor-core STGD.  YA/YB/YC are (Yq, scales) pairs from quantize_samples
    (pass the same pair three times for symmetric views)."""
    k = V.shape[0]
    n = YA[1].shape[0]  # the scales: one per sample (Yq has 2 n rows for PREC_FP8X2)
    _need(V, torch.float32, (k, k), "V")
    _need(ybar3, torch.float64, (3, k), "ybar3")
    if perm is not None:
        _need(perm, torch.int32, (epochs, n), "perm")
    steps = ((n + b - 1) // b) * epochs
    snaps = None
    if snapshot_every:
        snaps = torch.empty(max(steps // snapshot_every, 1), k, k, dtype=torch.float32,
                            device=V.device)
    ws = _ws(_lib.otm_sgd_run_lp_workspace(), V.device)
    _check(_lib.otm_sgd_run_lp(_ptr(V), _ptr(YA[0]), _ptr(YB[0]), _ptr(YC[0]), _ptr(YA[1]),
                               _ptr(YB[1]), _ptr(YC[1]), n, k, _ptr(ybar3), _ptr(perm),
                               int(epochs), int(b), float(beta0), float(theta), float(alpha0),
                               int(precision), int(snapshot_every), _ptr(snaps), _ptr(ws),
                               ws.numel(), _stream()))
    return snaps


class SgdBatch:
    """Many independent tensor-core STGD chains in one persistent launch.

    problems: list of dicts with keys Yq, scales (from quantize_samples), ybar3
    (3 x k float64), V (restarts x k x k float32, updated in place), perm
    (epochs x n int32 or None), epochs, b, beta0, theta, alpha0.  The
    referenced tensors must stay alive while the batch is used.  ``launch()``
    is asynchronous and capturable in a CUDA graph; ``check()`` synchronises
    and raises if a device wait timed out."""

    def __init__(self, problems, precision: int, cluster: int = 0):
        arr = (OtmProblem * len(problems))()
        dev = None
        for i, p in enumerate(problems):
            V = p["V"]
            r, k, k2 = V.shape
            if k != k2:
                raise ValueError("V must be restarts x k x k")
            n = p["Yq"].shape[0]
            _need(V, torch.float32, (r, k, k), "V")
            _need(p["ybar3"], torch.float64, (3, k), "ybar3")
            if p.get("perm") is not None:
                _need(p["perm"], torch.int32, (p["epochs"], n), "perm")
            arr[i] = OtmProblem(n, k, int(p["b"]), int(p["epochs"]), _ptr(p["Yq"]),
                                _ptr(p.get("scales")), _ptr(p.get("perm")), _ptr(p["ybar3"]),
                                _ptr(V), r, float(p["beta0"]), float(p["theta"]),
                                float(p["alpha0"]))
            dev = V.device
        nitems = sum(int(p["V"].shape[0]) for p in problems)
        self.ws = _ws(_lib.otm_sgd_batched_workspace(nitems), dev)
        self.plan = OtmBatchPlan()
        self._problems = arr
        _check(_lib.otm_sgd_batched_prepare(arr, len(problems), int(precision), int(cluster),
                                            _ptr(self.ws), self.ws.numel(),
                                            ctypes.byref(self.plan), _stream()))

    @property
    def cluster(self) -> int:
        return int(self.plan.cluster)

    @property
    def nitems(self) -> int:
        return int(self.plan.nitems)

    def launch(self) -> None:
        _check(_lib.otm_sgd_batched_launch(ctypes.byref(self.plan), _stream()))

    def check(self) -> None:
        _check(_lib.otm_sgd_batched_check(ctypes.byref(self.plan), _stream()))


# ---- learned warm start -------------------------------------------------

def gemm_bf16(A, B, epilogue: int = 0, alpha: float = 1.0, bias=None, want_c: bool = True,
              want_h: bool = False):
    """C = alpha A B^T (+ bias, GELU) for BF16 A (batch x M x K or M x K) and B
    (batch x N x K or N x K).  Returns (C float32 or None, H bfloat16 or None)."""
    batched = A.dim() == 3
    A3 = A if batched else A.unsqueeze(0)
    B3 = B if batched else B.unsqueeze(0)
    nb, M, K = A3.shape
    N = B3.shape[1]
    _need(A3, torch.bfloat16, (nb, M, K), "A")
    _need(B3, torch.bfloat16, (nb, N, K), "B")
    C = torch.empty(nb, M, N, dtype=torch.float32, device=A.device) if want_c else None
    H = torch.empty(nb, M, N, dtype=torch.bfloat16, device=A.device) if want_h else None
    ws = _ws(_lib.otm_gemm_bf16_workspace(), A.device)
    _check(_lib.otm_gemm_bf16(_ptr(A3), _ptr(B3), M, N, K, nb, K, K, M * K, N * K, int(epilogue),
                              float(alpha), _ptr(bias), _ptr(C), N, M * N, _ptr(H), N, M * N,
                              _ptr(ws), ws.numel(), _stream()))
    _check(_lib.otm_ws_check(_ptr(ws), _stream()))
    if not batched:
        C = None if C is None else C[0]
        H = None if H is None else H[0]
    return C, H


def gram_schmidt(M):
    nb, k, _ = M.shape
    _need(M, torch.float32, (nb, k, k), "M")
    U = torch.empty_like(M)
    R = torch.empty_like(M)
    _check(_lib.otm_gram_schmidt(_ptr(M), nb, k, _ptr(U), _ptr(R), _stream()))
    return U, R


def gram_schmidt_backward(U, R, dU):
    nb, k, _ = U.shape
    for t, nm in ((U, "U"), (R, "R"), (dU, "dU")):
        _need(t, torch.float32, (nb, k, k), nm)
    dM = torch.empty_like(U)
    _check(_lib.otm_gram_schmidt_backward(_ptr(U), _ptr(R), _ptr(dU), nb, k, _ptr(dM), _stream()))
    return dM


def ws_loss_grad(U, Ustar, lam, scale: float = 1.0):
    nb, k, _ = U.shape
    _need(U, torch.float32, (nb, k, k), "U")
    _need(Ustar, torch.float32, (nb, k, k), "Ustar")
    _need(lam, torch.float32, (nb, k), "lam")
    loss = torch.empty(nb, dtype=torch.float32, device=U.device)
    dU = torch.empty_like(U)
    _check(_lib.otm_ws_loss_grad(_ptr(U), _ptr(Ustar), _ptr(lam), nb, k, float(scale), _ptr(loss),
                                 _ptr(dU), _stream()))
    return loss, dU


def ws_generate(m, alpha, n: int, seed: int, first: int = 0):
    """Samples (nb x n x k float32) of whitened exact-mixture LDA instances."""
    nb, k, _ = m.shape
    _need(m, torch.float32, (nb, k, k), "m")
    _need(alpha, torch.float32, (nb, k), "alpha")
    Y = torch.empty(nb, n, k, dtype=torch.float32, device=m.device)
    _check(_lib.otm_ws_generate(_ptr(m), _ptr(alpha), nb, int(n), k, int(seed), int(first),
                                _ptr(Y), _stream()))
    return Y


def ws_sketch(Y, alpha0, thetas, want_s: bool = True):
    """(S: nb x J x k x k float32 or None, x16: nb x J k^2 bfloat16)."""
    nb, n, k = Y.shape
    J = thetas.shape[0]
    _need(Y, torch.float32, (nb, n, k), "Y")
    _need(alpha0, torch.float64, (nb,), "alpha0")
    _need(thetas, torch.float32, (J, k), "thetas")
    S = torch.empty(nb, J, k, k, dtype=torch.float32, device=Y.device) if want_s else None
    x16 = torch.empty(nb, J * k * k, dtype=torch.bfloat16, device=Y.device)
    ws = _ws(_lib.otm_ws_sketch_workspace(nb, n, k, J), Y.device)
    _check(_lib.otm_ws_sketch(_ptr(Y), nb, n, k, _ptr(alpha0), _ptr(thetas), J, _ptr(S), _ptr(x16),
                              _ptr(ws), ws.numel(), _stream()))
    _check(_lib.otm_ws_check(_ptr(ws), _stream()))
    return S, x16


def ws_canonicalize(S):
    """(E: nb x k x k, evals: nb x k, x16: nb x J k^2 bfloat16) of the sketches
    S (nb x J x k x k)."""
    nb, J, k, _ = S.shape
    _need(S, torch.float32, (nb, J, k, k), "S")
    E = torch.empty(nb, k, k, dtype=torch.float32, device=S.device)
    ev = torch.empty(nb, k, dtype=torch.float32, device=S.device)
    x16 = torch.empty(nb, J * k * k, dtype=torch.bfloat16, device=S.device)
    _check(_lib.otm_ws_canonicalize(_ptr(S), nb, k, J, _ptr(E), _ptr(ev), _ptr(x16), _stream()))
    return E, ev, x16


def ws_rotate(E, U, transpose: bool = False):
    nb, k, _ = E.shape
    _need(E, torch.float32, (nb, k, k), "E")
    _need(U, torch.float32, (nb, k, k), "U")
    out = torch.empty_like(U)
    _check(_lib.otm_ws_rotate(_ptr(E), _ptr(U), nb, k, int(bool(transpose)), _ptr(out), _stream()))
    return out


def ws_init_components(U0, Y, alpha0, theta: float):
    nb, n, k = Y.shape
    _need(U0, torch.float32, (nb, k, k), "U0")
    _need(alpha0, torch.float64, (nb,), "alpha0")
    V0 = torch.empty(nb, k, k, dtype=torch.float32, device=Y.device)
    ws = _ws(_lib.otm_ws_init_workspace(nb, n, k), Y.device)
    _check(_lib.otm_ws_init_components(_ptr(U0), _ptr(Y), nb, n, k, _ptr(alpha0), float(theta),
                                       _ptr(V0), _ptr(ws), ws.numel(), _stream()))
    return V0


class Mlp:
    """Warm-start network: FP32 master parameters (same order as
    otm_mlp_param_count), BF16 copies, gradient and Adam moments on the GPU."""

    def __init__(self, d_in: int, width: int, d_out: int, params, device="cuda"):
        self.d_in, self.width, self.d_out = d_in, width, d_out
        P = int(_lib.otm_mlp_param_count(d_in, width, d_out))
        self.p = torch.as_tensor(params, dtype=torch.float32).reshape(-1).to(device).contiguous()
        if self.p.numel() != P:
            raise ValueError(f"expected {P} parameters, got {self.p.numel()}")
        self.p16 = torch.empty(P, dtype=torch.bfloat16, device=device)
        self.w2t16 = torch.empty(width * width, dtype=torch.bfloat16, device=device)
        self.w3t16 = torch.empty(width * d_out, dtype=torch.bfloat16, device=device)
        self.grad = torch.zeros(P, dtype=torch.float32, device=device)
        self.m = torch.zeros(P, dtype=torch.float32, device=device)
        self.v = torch.zeros(P, dtype=torch.float32, device=device)
        self.t = 0
        self.desc = OtmMlp(d_in, width, d_out, _ptr(self.p), _ptr(self.p16), _ptr(self.w2t16),
                           _ptr(self.w3t16), _ptr(self.grad), _ptr(self.m), _ptr(self.v))
        self._ws = {}
        _check(_lib.otm_mlp_sync_weights(ctypes.byref(self.desc), _stream()))

    def _workspace(self, kind: str, batch: int):
        key = (kind, batch)
        if key not in self._ws:
            fn = _lib.otm_mlp_workspace if kind == "mlp" else _lib.otm_ws_train_workspace
            self._ws[key] = _ws(fn(ctypes.byref(self.desc), batch), self.p.device)
        return self._ws[key]

    def forward(self, x16):
        B = x16.shape[0]
        _need(x16, torch.bfloat16, (B, self.d_in), "x16")
        out = torch.empty(B, self.d_out, dtype=torch.float32, device=x16.device)
        ws = self._workspace("mlp", B)
        _check(_lib.otm_mlp_forward(ctypes.byref(self.desc), _ptr(x16), B, _ptr(out), _ptr(ws),
                                    ws.numel(), _stream()))
        return out

    def backward(self, x16, dout):
        """net.grad from dL/dout; uses the cache of the last forward(x16)."""
        B = x16.shape[0]
        _need(dout, torch.float32, (B, self.d_out), "dout")
        ws = self._workspace("mlp", B)
        _check(_lib.otm_mlp_backward(ctypes.byref(self.desc), _ptr(x16), B, _ptr(dout), _ptr(ws),
                                     ws.numel(), _stream()))
        _check(_lib.otm_ws_check(_ptr(ws), _stream()))
        return self.grad

    def adam(self, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.t += 1
        _check(_lib.otm_adam_step(ctypes.byref(self.desc), float(lr), float(b1), float(b2),
                                  float(eps), self.t, _stream()))

    def train_step(self, x16, Ustar, lam, k: int, lr: float):
        """One training step; returns the per-instance losses (device)."""
        B = x16.shape[0]
        _need(x16, torch.bfloat16, (B, self.d_in), "x16")
        _need(Ustar, torch.float32, (B, k, k), "Ustar")
        _need(lam, torch.float32, (B, k), "lam")
        loss = torch.empty(B, dtype=torch.float32, device=x16.device)
        ws = self._workspace("train", B)
        self.t += 1
        _check(_lib.otm_ws_train_step(ctypes.byref(self.desc), _ptr(x16), _ptr(Ustar), _ptr(lam),
                                      B, k, float(lr), self.t, _ptr(loss), _ptr(ws), ws.numel(),
                                      _stream()))
        return loss

    def infer(self, x16, k: int):
        B = x16.shape[0]
        _need(x16, torch.bfloat16, (B, self.d_in), "x16")
        U0 = torch.empty(B, k, k, dtype=torch.float32, device=x16.device)
        ws = self._workspace("train", B)
        _check(_lib.otm_ws_infer(ctypes.byref(self.desc), _ptr(x16), B, k, _ptr(U0), _ptr(ws),
                                 ws.numel(), _stream()))
        return U0

    def check(self, batch: int) -> None:
        for key, ws in self._ws.items():
            if key[1] == batch:
                _check(_lib.otm_ws_check(_ptr(ws), _stream()))


def unwhiten(V, Q, Cp, theta: float, normalize: bool) -> dict:
    k = V.shape[0]
    d, kt = Q.shape
    _need(V, torch.float32, (k, k), "V")
    _need(Q, torch.float32, (d, kt), "Q")
    _need(Cp, torch.float64, (kt, k), "Cp")
    dev = V.device
    o = {"comps": torch.empty(d, k, dtype=torch.float64, device=dev),
         "lambda": torch.empty(k, dtype=torch.float64, device=dev),
         "alpha_hat": torch.empty(k, dtype=torch.float64, device=dev)}
    ws = _ws(_lib.otm_unwhiten_workspace(d, k, kt), dev)
    _check(_lib.otm_unwhiten(_ptr(V), k, _ptr(Q), d, kt, _ptr(Cp), float(theta), int(bool(normalize)),
                             _ptr(o["comps"]), _ptr(o["lambda"]), _ptr(o["alpha_hat"]), _ptr(ws),
                             ws.numel(), _stream()))
    return o


def recon_error(V, U_true, lam_true, theta: float):
    """U_true: k x k with U_true[j] = unit component j (column-major storage)."""
    k = V.shape[0]
    _need(V, torch.float32, (k, k), "V")
    _need(U_true, torch.float64, (k, k), "U_true")
    _need(lam_true, torch.float64, (k,), "lam_true")
    err = torch.empty(1, dtype=torch.float64, device=V.device)
    ws = _ws(_lib.otm_recon_error_workspace(k), V.device)
    _check(_lib.otm_recon_error(_ptr(V), k, float(theta), _ptr(U_true), _ptr(lam_true), _ptr(err),
                                _ptr(ws), ws.numel(), _stream()))
    return err


def membership(Y, V, theta: float, tau: float = float("-inf")):
    """otm_membership: Pi_hat (k x n float32) from the view-A samples Y (n x k)
    and the components V (k x k, V[i] = component i)."""
    n, k = Y.shape
    _need(Y, torch.float32, (n, k), "Y")
    _need(V, torch.float32, (k, k), "V")
    out = torch.empty(k, n, dtype=torch.float32, device=Y.device)
    ws = _ws(_lib.otm_membership_workspace(k), Y.device)
    _check(_lib.otm_membership(_ptr(Y), n, k, _ptr(V), float(theta), float(tau), _ptr(out),
                               _ptr(ws), ws.numel(), _stream()))
    return out


def pvalue_match(Pi_hat, Pi, threshold: float = 0.01) -> dict:
    """otm_pvalue_match: p-values, l1 distances, recovery ratio and average
    error of Pi_hat (k_hat x n) against Pi (k x n), both float32."""
    k_hat, n = Pi_hat.shape
    k = Pi.shape[0]
    _need(Pi_hat, torch.float32, (k_hat, n), "Pi_hat")
    _need(Pi, torch.float32, (k, n), "Pi")
    dev = Pi_hat.device
    o = {"pvalues": torch.empty(k_hat, k, dtype=torch.float64, device=dev),
         "l1": torch.empty(k_hat, k, dtype=torch.float64, device=dev),
         "scores": torch.empty(2, dtype=torch.float64, device=dev)}
    ws = _ws(_lib.otm_pvalue_match_workspace(k_hat, k), dev)
    _check(_lib.otm_pvalue_match(_ptr(Pi_hat), k_hat, _ptr(Pi), k, n, float(threshold),
                                 _ptr(o["pvalues"]), _ptr(o["l1"]), _ptr(o["scores"]), _ptr(ws),
                                 ws.numel(), _stream()))
    return o


ENTRY_POINTS = tuple(_SIGS)
