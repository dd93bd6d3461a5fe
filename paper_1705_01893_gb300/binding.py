"""Thin ctypes binding of ``libmm.so`` (C ABI in ``include/mm.h``).

Argument marshalling only: torch tensors provide device memory and the CUDA stream; every
step of the solver runs in the library's kernels.  There is no CPU fallback: if the
library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmm.so")

MM_OK, MM_ERR_ARG, MM_ERR_CUDA, MM_ERR_NOMEM, MM_ERR_TIMEOUT, MM_ERR_STATE, MM_ERR_SINGULAR, \
    MM_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
MM_W_F32, MM_W_F16 = 0, 1
MM_FP32_MIXED = 0
MM_STAGE_LOAD, MM_STAGE_GATHER_FFT, MM_STAGE_FILTER, MM_STAGE_IFFT_BIN, MM_STAGE_MAP, MM_STAGE_FUSED = range(6)

_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_szp = ctypes.POINTER(ctypes.c_size_t)
_ip = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes); mirrors include/mm.h
SIGNATURES = {
    "mm_plan_workspace_size": (ctypes.c_int, [ctypes.c_int, _i64p, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_int, _szp]),
    "mm_plan_pointing": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64p, _vp, _vp, _vp,
                                        ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                        _vp, ctypes.c_size_t, _vp]),
    "mm_set_noise_psd": (ctypes.c_int, [_vp, _vp, _dp, _dp, _vp, _vp]),
    "mm_lambda_max": (ctypes.c_int, [_vp, _dp, _vp]),
    "mm_messenger_iterate": (ctypes.c_int, [_vp, _dp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
    "mm_plan_batches": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "mm_messenger_graph": (ctypes.c_int, [_vp, _dp, ctypes.c_int, _vp, _vp, _vp]),
    "mm_messenger_stage": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp, _vp,
                                          _vp]),
    "mm_plain_work_bytes": (ctypes.c_int, [_vp, _szp]),
    "mm_messenger_plain_fp64": (ctypes.c_int, [_vp, _vp, _dp, ctypes.c_int, _vp, _vp, _vp,
                                               ctypes.c_size_t, _vp]),
    "mm_adjoint_work_bytes": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _szp]),
    "mm_messenger_adjoint": (ctypes.c_int, [_vp, _dp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int,
                                            _vp, ctypes.c_size_t, _vp]),
    "mm_messenger_forward_ckpt": (ctypes.c_int, [_vp, _dp, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                                 _vp]),
    "mm_messenger_adjoint_ckpt": (ctypes.c_int, [_vp, _dp, ctypes.c_int, _vp, _vp, _vp, _vp,
                                                 ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "mm_plan_fault_flags": (ctypes.c_int, [_vp, _ip, _vp]),
    "mm_plan_set_wait_policy": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "mm_check_bounded_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _ip, _vp]),
    "mm_fused_item_list": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip,
                                          ctypes.c_int, _ip]),
    "mm_plan_fused_batches": (ctypes.c_int, [_vp, _ip]),
    "mm_pcg_state_bytes": (ctypes.c_int, [_vp, _szp]),
    "mm_pcg_iterate": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp]),
    "mm_chi2": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp, _vp]),
    "mm_chi2_modes": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    "mm_autotune": (ctypes.c_int, [_vp, _vp]),
    "mm_plan_workspace_size_composite": (ctypes.c_int, [ctypes.c_int, _i64p, ctypes.c_int64,
                                                        ctypes.c_int, ctypes.c_int, _szp]),
    "mm_plan_composite": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64p, _vp, _vp, _vp,
                                         ctypes.c_float, _vp, _vp, _vp, ctypes.c_float,
                                         ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_double, _vp, ctypes.c_size_t, _vp]),
    "mm_messenger_md_bytes": (ctypes.c_int, [_vp, ctypes.c_int, _szp]),
    "mm_messenger_iterate_md": (ctypes.c_int, [_vp, _dp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "mm_messenger_adaptive": (ctypes.c_int, [_vp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]),
    "mm_set_tune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "mm_get_tune": (ctypes.c_int, [_vp, _ip, _ip, _ip, _ip]),
    "mm_apply_pointing": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mm_apply_pointing_T": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mm_rfft": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mm_plan_maps": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "mm_binned_map_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int, ctypes.c_double, _vp,
                                             _vp]),
    "mm_plan_destroy": (None, [_vp]),
    "mm_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmm.so (built by ``paper_1705_01893_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with paper_1705_01893_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MMError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} -> {code}: {msg}")
        self.code = code


def _check(fn: str, code: int):
    if code != MM_OK:
        raise MMError(fn, code, load().mm_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dptr(arr: Optional[np.ndarray]):
    if arr is None:
        return None
    arr = np.ascontiguousarray(arr, dtype=np.float64)
    return arr.ctypes.data_as(_dp), arr


class Plan:
    """A pointing plan plus noise model on one GPU.

    pix, cos2psi, sin2psi and the workspace are torch CUDA tensors owned by this object
    (the library keeps raw pointers to them for the plan's lifetime)."""

    def __init__(self, offsets: Sequence[int], pix, cos2psi, sin2psi, n_pix: int, ncomp: int,
                 rcond_min: float = 1e-3, stream=None, second=None):
        """second: None, or (pix_b, cos_b, sin_b, gain_a, gain_b) for a composite plan
        (App. B: P = gain_a P(pix, cos2psi, sin2psi) + gain_b P(pix_b, cos_b, sin_b))."""
        import torch
        lib = load()
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n_chunks = len(self.offsets) - 1
        self.n_pix, self.ncomp = int(n_pix), int(ncomp)
        if pix.dtype != torch.int32 or not pix.is_cuda:
            raise TypeError("pix must be an int32 CUDA tensor")
        self.pix = pix.contiguous()
        self.cos2psi = None if cos2psi is None else cos2psi.contiguous()
        self.sin2psi = None if sin2psi is None else sin2psi.contiguous()
        wd = MM_W_F32
        if self.cos2psi is not None and self.cos2psi.dtype == torch.float16:
            wd = MM_W_F16
        self.weight_dtype = wd
        nbytes = ctypes.c_size_t()
        offp = self.offsets.ctypes.data_as(_i64p)
        self.second = None
        if second is not None:
            pb, cb, sb, ga, gb = second
            self.second = (pb.contiguous(), None if cb is None else cb.contiguous(),
                           None if sb is None else sb.contiguous(), float(ga), float(gb))
            _check("mm_plan_workspace_size_composite", lib.mm_plan_workspace_size_composite(
                self.n_chunks, offp, self.n_pix, self.ncomp, wd, ctypes.byref(nbytes)))
        else:
            _check("mm_plan_workspace_size", lib.mm_plan_workspace_size(
                self.n_chunks, offp, self.n_pix, self.ncomp, wd, ctypes.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=pix.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self._ws_bytes = int(nbytes.value)
        self.device = pix.device
        h = _vp()
        if self.second is not None:
            pb, cb, sb, ga, gb = self.second
            _check("mm_plan_composite", lib.mm_plan_composite(
                ctypes.byref(h), self.n_chunks, offp, _ptr(self.pix), _ptr(self.cos2psi),
                _ptr(self.sin2psi), ga, _ptr(pb), _ptr(cb), _ptr(sb), gb, wd, self.n_pix,
                self.ncomp, float(rcond_min), self._ws_ptr, self._ws_bytes, _stream(stream)))
        else:
            _check("mm_plan_pointing", lib.mm_plan_pointing(
                ctypes.byref(h), self.n_chunks, offp, _ptr(self.pix), _ptr(self.cos2psi),
                _ptr(self.sin2psi), wd, self.n_pix, self.ncomp, float(rcond_min), self._ws_ptr,
                self._ws_bytes, _stream(stream)))
        self._h = h
        self._pcg_state = None

    # --------------------------------------------------------------------------- life
    def close(self):
        if getattr(self, "_h", None):
            load().mm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------------- set-up
    def set_noise(self, tod, params: Optional[np.ndarray] = None, psd=None,
                  tau: Optional[np.ndarray] = None, stream=None):
        """params: [n_chunks, 4] (sigma, fknee, alpha, fs) or psd: CUDA float64 tensor."""
        lib = load()
        pp = _dptr(None if params is None else np.asarray(params).reshape(-1))
        tp = _dptr(tau)
        _check("mm_set_noise_psd", lib.mm_set_noise_psd(
            self._h, _ptr(psd), pp[0] if pp else None, tp[0] if tp else None,
            _ptr(tod.contiguous()), _stream(stream)))

    def lambda_max(self, stream=None) -> float:
        out = ctypes.c_double()
        _check("mm_lambda_max", load().mm_lambda_max(self._h, ctypes.byref(out), _stream(stream)))
        return out.value

    # ---------------------------------------------------------------------- solvers
    def messenger(self, map_inout, lambdas, chi2_out=None, stream=None):
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        _check("mm_messenger_iterate", load().mm_messenger_iterate(
            self._h, lam.ctypes.data_as(_dp), len(lam), MM_FP32_MIXED, _ptr(map_inout),
            _ptr(chi2_out), _stream(stream)))

    def messenger_graph(self, map_inout, lambdas, chi2_out=None, stream=None):
        """Same as messenger(), replaying one captured CUDA graph per iteration."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        _check("mm_messenger_graph", load().mm_messenger_graph(
            self._h, lam.ctypes.data_as(_dp), len(lam), _ptr(map_inout), _ptr(chi2_out),
            _stream(stream)))

    def messenger_plain_fp64(self, map_inout, lambdas, chi2_out=None, tod=None, stream=None):
        """The plain FP64 single-launch-per-iteration messenger step (comparison bar); tod
        defaults to the data the plan was set up with (plan_from_synth keeps it)."""
        import torch
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        n = ctypes.c_size_t()
        _check("mm_plain_work_bytes", load().mm_plain_work_bytes(self._h, ctypes.byref(n)))
        if getattr(self, "_plain_work", None) is None or self._plain_work.numel() < n.value + 256:
            self._plain_work = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=self.device)
        wp = (self._plain_work.data_ptr() + 255) // 256 * 256
        tod = self.tod if tod is None else tod
        _check("mm_messenger_plain_fp64", load().mm_messenger_plain_fp64(
            self._h, _ptr(tod), lam.ctypes.data_as(_dp), len(lam), _ptr(map_inout),
            _ptr(chi2_out), wp, int(n.value), _stream(stream)))

    def fault_flags(self, stream=None) -> int:
        """Fault flags of the plan's kernels since the last call (then cleared); 0 = none."""
        f = ctypes.c_int()
        _check("mm_plan_fault_flags", load().mm_plan_fault_flags(self._h, ctypes.byref(f),
                                                                 _stream(stream)))
        return f.value

    def set_wait_policy(self, n_polls: int = 1 << 22, check_on_return: bool = False):
        """Poll limit of the fused launch's bounded waits and whether the solver calls
        synchronise and raise MMError(MM_ERR_TIMEOUT) when one of them ran out."""
        _check("mm_plan_set_wait_policy", load().mm_plan_set_wait_policy(
            self._h, int(n_polls), int(bool(check_on_return))))

    def n_fused_batches(self) -> int:
        n = ctypes.c_int()
        _check("mm_plan_fused_batches", load().mm_plan_fused_batches(self._h, ctypes.byref(n)))
        return n.value

    def n_batches(self) -> int:
        n = ctypes.c_int()
        _check("mm_plan_batches", load().mm_plan_batches(self._h, ctypes.byref(n)))
        return n.value

    def stage(self, stage: int, batch: int = 0, lam: float = 1.0, map_inout=None, chi2_slot=None,
              stream=None):
        _check("mm_messenger_stage", load().mm_messenger_stage(
            self._h, int(stage), int(batch), float(lam), _ptr(map_inout), _ptr(chi2_slot),
            _stream(stream)))

    def adjoint(self, lambdas, map_in, grad_map_out, grad_tod, grad_theta=None,
                ckpt_every: int = 10, stream=None):
        """dL/dd (and dL/dtheta) through len(lambdas) iterations from map_in, given dL/dm_K."""
        import torch
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        n = ctypes.c_size_t()
        _check("mm_adjoint_work_bytes", load().mm_adjoint_work_bytes(self._h, len(lam), int(ckpt_every),
                                                                     ctypes.byref(n)))
        work = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=self.device)
        wp = (work.data_ptr() + 255) // 256 * 256
        _check("mm_messenger_adjoint", load().mm_messenger_adjoint(
            self._h, lam.ctypes.data_as(_dp), len(lam), _ptr(map_in), _ptr(grad_map_out),
            _ptr(grad_tod), _ptr(grad_theta), int(ckpt_every), wp, int(n.value), _stream(stream)))
        self._adj_work = work   # keep alive until the stream has run the call

    def forward_ckpt(self, map_inout, lambdas, ckpt_every: int = 10, stream=None):
        """len(lambdas) messenger iterations on map_inout; returns the checkpoints m_0, m_E,
        ... (E = ckpt_every) as a CUDA float64 tensor [ceil(K / E), n_pix, ncomp]."""
        import torch
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        nseg = (len(lam) + ckpt_every - 1) // ckpt_every
        ckpt = torch.empty((nseg,) + tuple(map_inout.shape), dtype=torch.float64,
                           device=self.device)
        _check("mm_messenger_forward_ckpt", load().mm_messenger_forward_ckpt(
            self._h, lam.ctypes.data_as(_dp), len(lam), _ptr(map_inout), int(ckpt_every),
            _ptr(ckpt), _stream(stream)))
        return ckpt

    def adjoint_ckpt(self, lambdas, ckpt, grad_map_out, grad_tod, grad_theta=None,
                     ckpt_every: int = 10, stream=None):
        """The backward of forward_ckpt: dL/dd (and dL/dtheta) from its checkpoints."""
        import torch
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        n = ctypes.c_size_t()
        _check("mm_adjoint_work_bytes", load().mm_adjoint_work_bytes(self._h, len(lam), int(ckpt_every),
                                                                     ctypes.byref(n)))
        work = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=self.device)
        wp = (work.data_ptr() + 255) // 256 * 256
        _check("mm_messenger_adjoint_ckpt", load().mm_messenger_adjoint_ckpt(
            self._h, lam.ctypes.data_as(_dp), len(lam), _ptr(ckpt), _ptr(grad_map_out),
            _ptr(grad_tod), _ptr(grad_theta), int(ckpt_every), wp, int(n.value), _stream(stream)))
        self._adj_work = work   # keep alive until the stream has run the call

    def pcg_state(self):
        import torch
        if self._pcg_state is None:
            n = ctypes.c_size_t()
            _check("mm_pcg_state_bytes", load().mm_pcg_state_bytes(self._h, ctypes.byref(n)))
            self._pcg_state_t = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=self.device)
            self._pcg_state = (self._pcg_state_t.data_ptr() + 255) // 256 * 256
        return self._pcg_state

    def pcg(self, map_inout, n_iter: int, restart: bool = True, chi2_out=None, stream=None):
        st = self.pcg_state()
        _check("mm_pcg_iterate", load().mm_pcg_iterate(
            self._h, int(n_iter), _ptr(map_inout), st, int(bool(restart)), _ptr(chi2_out),
            _stream(stream)))

    def chi2(self, map_in, lam: float = 1.0, out=None, stream=None):
        import torch
        if out is None:
            out = torch.zeros(1, dtype=torch.float64, device=self.device)
        _check("mm_chi2", load().mm_chi2(self._h, _ptr(map_in), float(lam), _ptr(out),
                                         _stream(stream)))
        return out

    def chi2_modes(self, map_in, lam: float = 1.0, stream=None):
        """(total chi^2 [1], per-mode chi^2 [sum_c (n_c/2+1)]) as CUDA float64 tensors."""
        import torch
        n_modes = int(sum(int(self.offsets[c + 1] - self.offsets[c]) // 2 + 1
                          for c in range(self.n_chunks)))
        total = torch.zeros(1, dtype=torch.float64, device=self.device)
        modes = torch.empty(n_modes, dtype=torch.float64, device=self.device)
        _check("mm_chi2_modes", load().mm_chi2_modes(self._h, _ptr(map_in), float(lam), _ptr(total),
                                                     _ptr(modes), _stream(stream)))
        return total, modes

    def messenger_md(self, map_inout, lambdas, chi2_out=None, stream=None):
        """Map-sized form m' = m_d(lambda) + F(lambda) m over the schedule `lambdas` (m_d
        formed once per distinct lambda in a work buffer allocated here)."""
        import torch
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        n_lev = max(1, len(set(lam.tolist())))
        nb = ctypes.c_size_t()
        _check("mm_messenger_md_bytes", load().mm_messenger_md_bytes(self._h, n_lev, ctypes.byref(nb)))
        work = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device=self.device)
        wp = (work.data_ptr() + 255) // 256 * 256
        _check("mm_messenger_iterate_md", load().mm_messenger_iterate_md(
            self._h, lam.ctypes.data_as(_dp), len(lam), _ptr(map_inout), _ptr(chi2_out), wp,
            int(nb.value), _stream(stream)))
        self._md_work = work   # keep alive until the stream has run the call

    def messenger_adaptive(self, map_inout, levels, rel_tol: float, min_per_level: int = 2,
                           max_per_level: int = 20, max_iter: int = 400, stream=None):
        """Plateau-driven cooling in one graph launch; returns (chi2 [n], lambda [n], n) with
        n the iterations run (synchronises the stream to read n)."""
        import torch
        lv = np.ascontiguousarray(levels, dtype=np.float64)
        chi = torch.zeros(max_iter, dtype=torch.float64, device=self.device)
        lam = torch.zeros(max_iter, dtype=torch.float64, device=self.device)
        nd = torch.zeros(1, dtype=torch.int32, device=self.device)
        _check("mm_messenger_adaptive", load().mm_messenger_adaptive(
            self._h, lv.ctypes.data_as(_dp), len(lv), float(rel_tol), int(min_per_level),
            int(max_per_level), int(max_iter), _ptr(map_inout), _ptr(chi), _ptr(lam), _ptr(nd),
            _stream(stream)))
        torch.cuda.current_stream(self.device).synchronize() if stream is None else stream.synchronize()
        n = int(nd.item())
        return chi[:n], lam[:n], n

    def autotune(self, stream=None):
        """Measure and keep the fastest schedule of the general-length kernels."""
        _check("mm_autotune", load().mm_autotune(self._h, _stream(stream)))

    @property
    def tune(self):
        """(col_nb, col_threads, row_threads, radix_order) of the general-length kernels."""
        v = [ctypes.c_int() for _ in range(4)]
        _check("mm_get_tune", load().mm_get_tune(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_tune(self, col_nb, col_threads, row_threads, radix_order, stream=None):
        _check("mm_set_tune", load().mm_set_tune(self._h, int(col_nb), int(col_threads),
                                                 int(row_threads), int(radix_order),
                                                 _stream(stream)))

    # -------------------------------------------------------------------- operators
    def apply_pointing(self, map_in, tod_out, stream=None):
        _check("mm_apply_pointing", load().mm_apply_pointing(self._h, _ptr(map_in), _ptr(tod_out),
                                                             _stream(stream)))

    def apply_pointing_T(self, tod, acc_out, stream=None):
        _check("mm_apply_pointing_T", load().mm_apply_pointing_T(self._h, _ptr(tod), _ptr(acc_out),
                                                                 _stream(stream)))

    def rfft(self, tod, spec_out, stream=None):
        _check("mm_rfft", load().mm_rfft(self._h, _ptr(tod), _ptr(spec_out), _stream(stream)))

    def maps(self, hits=None, valid=None, weight=None, stream=None):
        _check("mm_plan_maps", load().mm_plan_maps(self._h, _ptr(hits), _ptr(valid), _ptr(weight),
                                                   _stream(stream)))


def plan_from_synth(s: dict, device="cuda:0", rcond_min: float = 1e-3, tau=None, stream=None):
    """Upload a synthetic-data dict (see ``synth``) and build a plan with its noise model
    (a composite plan when the dict has a second pointing component, ``pix_b``)."""
    import torch
    dev = torch.device(device)
    pix = torch.from_numpy(s["pix"]).to(dev)
    cos = None if s["cos"] is None else torch.from_numpy(s["cos"]).to(dev)
    sin = None if s["sin"] is None else torch.from_numpy(s["sin"]).to(dev)
    tod = torch.from_numpy(s["tod"]).to(dev)
    second = None
    if s.get("pix_b") is not None:
        cb, sb = s.get("cos_b"), s.get("sin_b")
        second = (torch.from_numpy(s["pix_b"]).to(dev),
                  None if cb is None else torch.from_numpy(cb).to(dev),
                  None if sb is None else torch.from_numpy(sb).to(dev),
                  s.get("gain_a", 1.0), s.get("gain_b", -1.0))
    plan = Plan(s["offsets"], pix, cos, sin, s["npix"], s["ncomp"], rcond_min, stream=stream,
                second=second)
    plan.set_noise(tod, params=s["params"], tau=tau, stream=stream)
    plan.tod = tod
    return plan


def binned_map_noalloc(pix, cos2psi, sin2psi, tod, n_pix: int, ncomp: int, map_out,
                       rcond_min: float = 1e-3, stream=None):
    """(P^T P)^-1 P^T d per pixel with no device allocation by the library (its scratch is a
    fixed device array of 2^18 pixels); for callers that must not allocate.  The tensors are
    checked here (types, sizes, contiguity, one CUDA device) before any pointer is passed,
    because the kernels trust the sizes they are given."""
    import torch
    n = int(pix.numel())
    ts = [t for t in (pix, cos2psi, sin2psi, tod, map_out) if t is not None]
    if not all(isinstance(t, torch.Tensor) for t in ts):
        raise TypeError("binned_map_noalloc: every array must be a torch tensor")
    if pix.dtype != torch.int32:
        raise TypeError("binned_map_noalloc: pix must be int32")
    if tod.dtype != torch.float32 or tod.numel() != n:
        raise ValueError("binned_map_noalloc: tod must be float32 with pix.numel() elements")
    if ncomp not in (1, 3):
        raise ValueError("binned_map_noalloc: ncomp must be 1 or 3")
    if map_out.dtype != torch.float64 or map_out.numel() < int(n_pix) * int(ncomp):
        raise ValueError("binned_map_noalloc: map_out must be float64 with >= n_pix * ncomp "
                         "elements")
    if (ncomp == 3) != (cos2psi is not None and sin2psi is not None):
        raise ValueError("binned_map_noalloc: cos2psi and sin2psi are given iff ncomp == 3")
    wd = MM_W_F32
    if ncomp == 3:
        if cos2psi.dtype != sin2psi.dtype or cos2psi.dtype not in (torch.float32, torch.float16):
            raise TypeError("binned_map_noalloc: cos2psi and sin2psi must both be float32 or "
                            "both float16")
        if cos2psi.numel() != n or sin2psi.numel() != n:
            raise ValueError("binned_map_noalloc: cos2psi and sin2psi need pix.numel() elements")
        wd = MM_W_F16 if cos2psi.dtype == torch.float16 else MM_W_F32
    if any(not t.is_cuda for t in ts) or len({t.device for t in ts}) != 1:
        raise ValueError("binned_map_noalloc: every tensor must be on one CUDA device")
    if any(not t.is_contiguous() for t in ts):
        raise ValueError("binned_map_noalloc: every tensor must be contiguous")
    _check("mm_binned_map_noalloc", load().mm_binned_map_noalloc(
        _ptr(pix), _ptr(cos2psi), _ptr(sin2psi), wd, _ptr(tod), n, int(n_pix),
        int(ncomp), float(rcond_min), _ptr(map_out), _stream(stream)))


def fused_item_list(m1: int, m2: int, count: int) -> np.ndarray:
    """The fused kernel's work list for `count` chunks of complex length m1 x m2, as an int
    array [n_items, 3] of (kind, chunk, index); host only."""
    n = ctypes.c_int()
    _check("mm_fused_item_list", load().mm_fused_item_list(m1, m2, count, None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, 3), dtype=np.int32)
    _check("mm_fused_item_list", load().mm_fused_item_list(
        m1, m2, count, out.ctypes.data_as(_ip), n.value, ctypes.byref(n)))
    return out


def check_bounded_wait(n_polls: int, flag_set: bool, stream=None) -> bool:
    """Run the fused kernel's bounded wait on a device flag (set beforehand or never);
    returns True when the wait ran out."""
    e = ctypes.c_int()
    _check("mm_check_bounded_wait", load().mm_check_bounded_wait(int(n_polls), int(bool(flag_set)),
                                                                 ctypes.byref(e), _stream(stream)))
    return bool(e.value)


def cooling_schedule(lam_max: float, levels: int, iters: int) -> np.ndarray:
    """One lambda = inf step, then `levels` geometric levels lam_max -> 1, `iters` each."""
    if levels == 1:
        lv = [1.0]
    else:
        lv = [lam_max ** ((levels - 1 - j) / (levels - 1)) for j in range(levels)]
    return np.array([math.inf] + [v for v in lv for _ in range(iters)])


def messenger_fn():
    """torch.autograd.Function running K cooled messenger iterations on the GPU, with the
    hand-written adjoint as its backward.  apply(plan, lambdas, map_in, tod, theta) ->
    m_K; gradients flow to tod (float32 [n]) and theta (float64 [n_chunks, 3] =
    sigma, f_knee, alpha), which must be the data and parameters the plan was set up with.
    When theta needs a gradient the forward keeps checkpoints every CKPT_EVERY iterations
    for the backward's recomputation; otherwise the backward needs no forward iterate."""
    import torch

    class MessengerFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, plan, lambdas, map_in, tod, theta):
            m = map_in.detach().clone()
            lam = np.asarray(lambdas, dtype=np.float64)
            ctx.plan, ctx.lambdas = plan, lam
            ctx.want_theta = bool(ctx.needs_input_grad[4])
            if ctx.want_theta:
                # checkpoints every CKPT_EVERY iterations, taken during this forward
                ctx.save_for_backward(plan.forward_ckpt(m, lam, MessengerFn.CKPT_EVERY))
            else:
                plan.messenger(m, lam)     # dL/dd needs no forward iterate
                ctx.save_for_backward(m)
            return m

        @staticmethod
        def backward(ctx, grad_m):
            (ckpt,) = ctx.saved_tensors
            plan = ctx.plan
            gt = torch.empty(int(plan.offsets[-1]), dtype=torch.float32, device=grad_m.device)
            gth = None
            if ctx.want_theta:
                gth = torch.empty(plan.n_chunks, 3, dtype=torch.float64, device=grad_m.device)
            plan.adjoint_ckpt(ctx.lambdas, ckpt, grad_m.contiguous().to(torch.float64), gt, gth,
                              ckpt_every=MessengerFn.CKPT_EVERY)
            return None, None, None, gt, gth

    MessengerFn.CKPT_EVERY = 10

    return MessengerFn
