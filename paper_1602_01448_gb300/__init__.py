"""Python binding of the GB300 RAAR ptychography library (``include/sharp.h``).

Thin ctypes marshalling over ``_lib/libsharp.so``: every entry point has the
same name as its C function and takes CUDA tensors (complex64 images, probes
and frames; float32 amplitudes; int32 positions; float64 scalar outputs).
All arithmetic runs in the library's CUDA kernels; PyTorch provides device
memory and the current stream.  There is no CPU fallback: importing the
package fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import torch

__all__ = [
    "SharpError", "lib_path", "Plan", "sharp_default_params", "sharp_version",
    "sharp_plan_create", "sharp_plan_destroy", "sharp_q_gather", "sharp_fourier_project",
    "sharp_overlap_project", "sharp_probe_update", "sharp_raar_init", "sharp_raar_step",
    "sharp_solution_error", "sharp_forward_amplitudes", "sharp_amp_loss",
    "sharp_amp_loss_backward", "AmpLoss", "amp_loss", "sharp_plan_set_profiling",
    "sharp_plan_kernel_times", "sharp_plan_status", "sharp_plan_set_wait_limit", "sharp_fourier_project_noalloc",
    "Batch",
    "SHARP_PROBE_CONSTRAINT_NONE", "SHARP_PROBE_CONSTRAINT_MASK", "SHARP_PROBE_CONSTRAINT_AMPLITUDE",
    "SHARP_PREC_FP32", "SHARP_PREC_FP16S", "SHARP_PREC_BF16X3", "PRECISIONS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "_lib", "libsharp.so")

SHARP_OK = 0
_ERRNAMES = {1: "INVALID_ARG", 2: "UNSUPPORTED_SIZE", 3: "CUDA", 4: "TIMEOUT", 5: "STATE"}


class SharpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sharp error {code} ({_ERRNAMES.get(code, '?')}): {msg}")
        self.code = code


class sharp_params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_float), ("wrap", ctypes.c_int), ("probe_every", ctypes.c_int),
                ("residual_every", ctypes.c_int), ("precision", ctypes.c_int)]


if not os.path.exists(lib_path):
    raise ImportError(f"{lib_path} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")

_lib = ctypes.CDLL(lib_path)
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def _decl(name, argtypes, restype=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = argtypes
    f.restype = restype
    return f


_lib_fns = {
    "sharp_last_error": ([], ctypes.c_char_p),
    "sharp_version": ([], ctypes.c_char_p),
    "sharp_default_params": ([ctypes.POINTER(sharp_params)], None),
    "sharp_plan_create": ([ctypes.POINTER(_P), _I, _I, _I, _I, _P, ctypes.POINTER(sharp_params), _P], _I),
    "sharp_plan_destroy": ([_P], _I),
    "sharp_q_gather": ([_P, _P, _P, _P, _P], _I),
    "sharp_fourier_project": ([_P, _P, _P, _P, _P, _P], _I),
    "sharp_overlap_project": ([_P, _P, _P, _P, _P, _P], _I),
    "sharp_probe_update": ([_P, _P, _P, _P, _P, _P], _I),
    "sharp_raar_init": ([_P, _P, _P, _P, _P, _P, _P], _I),
    "sharp_raar_step": ([_P, _P, _P, _P, _P, _P, _P, _I, _P], _I),
    "sharp_solution_error": ([_P, _P, _P, _P, _P, _P], _I),
    "sharp_forward_amplitudes": ([_P, _P, _P, _P, _P], _I),
    "sharp_amp_loss": ([_P, _P, _P, _P, _P, _P], _I),
    "sharp_amp_loss_backward": ([_P, _P, _P, _P, _D, _P, _P, _P], _I),
    "sharp_plan_set_profiling": ([_P, _I], _I),
    "sharp_plan_status": ([_P, _P], _I),
    "sharp_plan_set_wait_limit": ([_P, ctypes.c_longlong], _I),
    "sharp_plan_set_deterministic": ([_P, _I], _I),
    "sharp_raar_checkpoint": ([_P, _P, _P, ctypes.POINTER(_I), _P], _I),
    "sharp_raar_restore": ([_P, _P, _P, ctypes.POINTER(_I), _P], _I),
    "sharp_fourier_project_noalloc": ([_P, _P, _P, _P, _I, _I, _P], _I),
    "sharp_plan_set_probe_refinement": ([_P, _I, _P, _I, _P], _I),
    "sharp_probe_refine": ([_P, _P, _P, _P], _I),
    "sharp_probe_init_mean": ([_P, _P, ctypes.c_float, _P, _P], _I),
    "sharp_batch_create": ([ctypes.POINTER(_P), _I, ctypes.POINTER(_P)], _I),
    "sharp_batch_bind": ([_P, _I, _P, _P, _P, _P, _P, _P], _I),
    "sharp_batch_step": ([_P, _I, _P], _I),
    "sharp_batch_set_graphs": ([_P, _I], _I),
    "sharp_batch_tuned_grid": ([_P, _I], _I),
    "sharp_batch_tuned_shape": ([_P, _I, _P, _P, _P], _I),
    "sharp_batch_set_shape": ([_P, _I, _I, _I, _I], _I),
    "sharp_batch_status": ([_P, _P], _I),
    "sharp_batch_destroy": ([_P], _I),
    "sharp_plan_kernel_times": ([_P, _P, _P], _I),
}
_C = {name: _decl(name, *sig) for name, sig in _lib_fns.items()}


# sharp_params.precision: FP32 transforms, or the frame DFTs as tensor-core
# contractions (m = 128, 256): FP16 with per-frame power-of-two scaling, or BF16
# three-term split; FP32 accumulation in both.
SHARP_PREC_FP32 = 0
SHARP_PREC_FP16S = 1
SHARP_PREC_BF16X3 = 2
PRECISIONS = {"fp32": SHARP_PREC_FP32, "fp16s": SHARP_PREC_FP16S, "bf16x3": SHARP_PREC_BF16X3}

SHARP_PROBE_CONSTRAINT_NONE = 0
SHARP_PROBE_CONSTRAINT_MASK = 1
SHARP_PROBE_CONSTRAINT_AMPLITUDE = 2


def _check(code: int):
    if code != SHARP_OK:
        raise SharpError(code, _C["sharp_last_error"]().decode())


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t, dtype, name, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


def sharp_version() -> str:
    return _C["sharp_version"]().decode()


def sharp_default_params() -> sharp_params:
    p = sharp_params()
    _C["sharp_default_params"](ctypes.byref(p))
    return p


def sharp_plan_create(K, m, ny, nx, pos, params=None, stream=None) -> int:
    h = _P()
    prm = params if params is not None else sharp_default_params()
    _check(_C["sharp_plan_create"](ctypes.byref(h), K, m, ny, nx, _ptr(pos, torch.int32, "pos", (K, 2)),
                                   ctypes.byref(prm), _stream(stream)))
    return h.value


def sharp_plan_destroy(plan) -> None:
    _check(_C["sharp_plan_destroy"](plan))


def _c64(t, name, shape=None):
    return _ptr(t, torch.complex64, name, shape)


def _f32(t, name, shape=None):
    return _ptr(t, torch.float32, name, shape)


def _f64(t, name, shape=None):
    return _ptr(t, torch.float64, name, shape)


def sharp_q_gather(plan, obj, probe, frames, stream=None):
    _check(_C["sharp_q_gather"](plan, _c64(obj, "obj"), _c64(probe, "probe"), _c64(frames, "frames"), _stream(stream)))


def sharp_fourier_project(plan, z, amp, out, resid_sq=None, stream=None):
    _check(_C["sharp_fourier_project"](plan, _c64(z, "z"), _f32(amp, "amp"), _c64(out, "out"),
                                       _f64(resid_sq, "resid_sq"), _stream(stream)))


def sharp_overlap_project(plan, probe, z, obj_out, z_out=None, stream=None):
    _check(_C["sharp_overlap_project"](plan, _c64(probe, "probe"), _c64(z, "z"), _c64(obj_out, "obj_out"),
                                       _c64(z_out, "z_out"), _stream(stream)))


def sharp_probe_update(plan, obj, z, probe_old, probe_out, stream=None):
    _check(_C["sharp_probe_update"](plan, _c64(obj, "obj"), _c64(z, "z"), _c64(probe_old, "probe_old"),
                                    _c64(probe_out, "probe_out"), _stream(stream)))


def sharp_raar_init(plan, psi0, probe0, state_c, psi_y, psi, stream=None):
    _check(_C["sharp_raar_init"](plan, _c64(psi0, "psi0"), _c64(probe0, "probe0"), _c64(state_c, "state_c"),
                                 _c64(psi_y, "psi_y"), _c64(psi, "psi"), _stream(stream)))


def sharp_raar_step(plan, state_c, psi_y, psi, probe, amp, metrics, it, stream=None):
    _check(_C["sharp_raar_step"](plan, _c64(state_c, "state_c"), _c64(psi_y, "psi_y"), _c64(psi, "psi"),
                                 _c64(probe, "probe"), _f32(amp, "amp"), _f64(metrics, "metrics"), int(it),
                                 _stream(stream)))


def sharp_solution_error(plan, psi, psi_true, probe, out, stream=None):
    _check(_C["sharp_solution_error"](plan, _c64(psi, "psi"), _c64(psi_true, "psi_true"), _c64(probe, "probe"),
                                      _f64(out, "out"), _stream(stream)))


def sharp_forward_amplitudes(plan, obj, probe, amp_out, stream=None):
    _check(_C["sharp_forward_amplitudes"](plan, _c64(obj, "obj"), _c64(probe, "probe"), _f32(amp_out, "amp_out"),
                                          _stream(stream)))


def sharp_amp_loss(plan, obj, probe, amp, loss, stream=None):
    _check(_C["sharp_amp_loss"](plan, _c64(obj, "obj"), _c64(probe, "probe"), _f32(amp, "amp"),
                                _f64(loss, "loss"), _stream(stream)))


def sharp_amp_loss_backward(plan, obj, probe, amp, grad_scale, g_obj, g_probe=None, stream=None):
    _check(_C["sharp_amp_loss_backward"](plan, _c64(obj, "obj"), _c64(probe, "probe"), _f32(amp, "amp"),
                                         float(grad_scale), _c64(g_obj, "g_obj"), _c64(g_probe, "g_probe"),
                                         _stream(stream)))


KCLASSES = ("frame", "image", "probe", "illum", "other")


def sharp_fourier_project_noalloc(z, amp, out, resid_sq=None, stream=None) -> None:
    """P_a of explicit frames without any device allocation (no plan)."""
    K, m = int(z.shape[0]), int(z.shape[-1])
    _check(_C["sharp_fourier_project_noalloc"](_c64(z, "z"), _f32(amp, "amp"), _c64(out, "out"),
                                               _f64(resid_sq, "resid_sq"), K, m, _stream(stream)))


def sharp_plan_status(plan, stream=None) -> None:
    """Synchronise the stream; raise SharpError if a kernel flagged a failure."""
    _check(_C["sharp_plan_status"](plan, _stream(stream)))


def sharp_plan_set_wait_limit(plan, polls: int) -> None:
    _check(_C["sharp_plan_set_wait_limit"](plan, int(polls)))


def sharp_plan_set_profiling(plan, enable: bool) -> None:
    _check(_C["sharp_plan_set_profiling"](plan, int(bool(enable))))


def sharp_plan_kernel_times(plan):
    """Per kernel class: (total ms, launches) since the last call."""
    ms = (ctypes.c_double * 5)()
    cnt = (ctypes.c_int * 5)()
    _check(_C["sharp_plan_kernel_times"](plan, ms, cnt))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KCLASSES)}


class Plan:
    """Owns a ``sharp_plan`` and the RAAR state tensors of one scan."""

    def __init__(self, pos, m, shape, beta=0.75, wrap=False, probe_every=0, residual_every=1,
                 device="cuda", precision="fp32"):
        pos = torch.as_tensor(pos, dtype=torch.int32).to(device).contiguous()
        self.K = int(pos.shape[0])
        self.m = int(m)
        self.shape = (int(shape[0]), int(shape[1]))
        self.device = torch.device(device)
        prm = sharp_default_params()
        prm.beta = float(beta)
        prm.wrap = int(bool(wrap))
        prm.probe_every = int(probe_every)
        prm.residual_every = int(residual_every)
        prm.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.params = prm
        self.pos = pos
        self.handle = sharp_plan_create(self.K, self.m, self.shape[0], self.shape[1], pos, prm)
        self.c = self.psi_y = self.psi = None
        self.metrics = torch.zeros(4, dtype=torch.float64, device=self.device)
        self.iter = 0

    def close(self):
        if getattr(self, "handle", None):
            sharp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        """Raise SharpError if a kernel of this plan flagged a failure (a bounded
        wait gave up, or invalid amplitudes or probe were seen)."""
        _check(_C["sharp_plan_status"](self.handle, _stream(stream)))

    def set_deterministic(self, enable=True):
        """Gather the overlap sums in a fixed order (bit-identical steps)."""
        _check(_C["sharp_plan_set_deterministic"](self.handle, int(bool(enable))))

    def checkpoint(self):
        """Everything needed to resume the reconstruction (host copies)."""
        pc = torch.empty((self.m, self.m), dtype=torch.complex64, device=self.device)
        pf = torch.empty_like(pc)
        info = (_I * 4)()
        _check(_C["sharp_raar_checkpoint"](self.handle, _c64(pc, "probe_cur"), _c64(pf, "probe_form"), info,
                                           _stream()))
        torch.cuda.synchronize(self.device)
        return {"c": self.c.cpu(), "psi_y": self.psi_y.cpu(), "psi": self.psi.cpu(), "probe": self.probe.cpu(),
                "probe_cur": pc.cpu(), "probe_form": pf.cpu(), "info": list(info), "iter": self.iter}

    def restore(self, ckpt):
        """Continue from checkpoint() of a plan over the same scan."""
        dev = self.device
        self.c = ckpt["c"].to(dev).contiguous()
        self.psi_y = ckpt["psi_y"].to(dev).contiguous()
        self.psi = ckpt["psi"].to(dev).contiguous()
        self.probe = ckpt["probe"].to(dev).contiguous()
        info = (_I * 4)(*ckpt["info"])
        pc = ckpt["probe_cur"].to(dev).contiguous()
        pf = ckpt["probe_form"].to(dev).contiguous()
        _check(_C["sharp_raar_restore"](self.handle, _c64(pc, "probe_cur"), _c64(pf, "probe_form"), info, _stream()))
        torch.cuda.synchronize(dev)   # the copies out of pc and pf are done
        self.iter = int(ckpt["iter"])

    def set_wait_limit(self, polls=-1):
        """Poll limit of the frame passes' bounded waits (-1: default, 0: give up at once)."""
        _check(_C["sharp_plan_set_wait_limit"](self.handle, int(polls)))

    # ---------------------------------------------------------- operators
    def q_gather(self, obj, probe):
        out = torch.empty((self.K, self.m, self.m), dtype=torch.complex64, device=self.device)
        sharp_q_gather(self.handle, obj, probe, out)
        return out

    def fourier_project(self, z, amp, out=None):
        out = torch.empty_like(z) if out is None else out
        r = torch.zeros(1, dtype=torch.float64, device=self.device)
        sharp_fourier_project(self.handle, z, amp, out, r)
        return out, r

    def overlap_project(self, probe, z, want_frames=True):
        obj = torch.empty(self.shape, dtype=torch.complex64, device=self.device)
        zo = torch.empty_like(z) if want_frames else None
        sharp_overlap_project(self.handle, probe, z, obj, zo)
        return obj, zo

    def probe_update(self, obj, z, probe_old):
        out = torch.empty_like(probe_old)
        sharp_probe_update(self.handle, obj, z, probe_old, out)
        return out

    def set_probe_refinement(self, mask=None, amplitude=None, center=False, stream=None):
        """What follows each probe update (Sec. 2.2 step 7): the Fourier mask
        if given, else the Fourier amplitudes if given, then the centring."""
        kind, vals = SHARP_PROBE_CONSTRAINT_NONE, None
        if mask is not None:
            kind, vals = SHARP_PROBE_CONSTRAINT_MASK, mask
        elif amplitude is not None:
            kind, vals = SHARP_PROBE_CONSTRAINT_AMPLITUDE, amplitude
        ptr = None if vals is None else _f32(vals, "values", (self.m, self.m))
        _check(_C["sharp_plan_set_probe_refinement"](self.handle, kind, ptr, int(bool(center)), _stream(stream)))

    def probe_refine(self, probe, out=None):
        out = torch.empty_like(probe) if out is None else out
        _check(_C["sharp_probe_refine"](self.handle, _c64(probe, "probe", (self.m, self.m)),
                                        _c64(out, "probe_out", (self.m, self.m)), _stream()))
        return out

    def probe_init_mean(self, amp, threshold=0.0):
        out = torch.empty((self.m, self.m), dtype=torch.complex64, device=self.device)
        _check(_C["sharp_probe_init_mean"](self.handle, _f32(amp, "amp", (self.K, self.m, self.m)),
                                           float(threshold), _c64(out, "probe_out"), _stream()))
        return out

    def forward_amplitudes(self, obj, probe):
        out = torch.empty((self.K, self.m, self.m), dtype=torch.float32, device=self.device)
        sharp_forward_amplitudes(self.handle, obj, probe, out)
        return out

    def solution_error(self, psi, psi_true, probe):
        out = torch.zeros(2, dtype=torch.float64, device=self.device)
        sharp_solution_error(self.handle, psi, psi_true, probe, out)
        return out

    # ---------------------------------------------------------- RAAR
    def raar_init(self, psi0, probe0):
        self.c = torch.empty((self.K, self.m, self.m), dtype=torch.complex64, device=self.device)
        self.psi_y = torch.empty(self.shape, dtype=torch.complex64, device=self.device)
        self.psi = torch.empty(self.shape, dtype=torch.complex64, device=self.device)
        self.probe = torch.empty((self.m, self.m), dtype=torch.complex64, device=self.device)
        sharp_raar_init(self.handle, psi0, probe0, self.c, self.psi_y, self.psi)
        self.probe.copy_(probe0)
        self.iter = 0

    def raar_step(self, amp, metrics=True):
        self.iter += 1
        sharp_raar_step(self.handle, self.c, self.psi_y, self.psi, self.probe, amp,
                        self.metrics if metrics else None, self.iter)
        return self.metrics if metrics else None


class Batch:
    """Independent scans stepped together by ``sharp_batch_step``: one
    persistent frame-pass launch per frame size, each step schedule recorded
    as a CUDA graph.  ``plans`` are ``Plan`` objects after ``raar_init``,
    ``amps`` their measured amplitudes; ``metrics`` of each plan are filled as
    by ``Plan.raar_step``."""

    def __init__(self, plans, amps, use_graphs=True):
        self.plans = list(plans)
        self.amps = list(amps)
        if len(self.amps) != len(self.plans):
            raise ValueError("one amplitude tensor per plan")
        arr = (_P * len(self.plans))(*[p.handle for p in self.plans])
        h = _P()
        _check(_C["sharp_batch_create"](ctypes.byref(h), len(self.plans), arr))
        self.handle = h.value
        _check(_C["sharp_batch_set_graphs"](self.handle, int(bool(use_graphs))))
        for i, (p, a) in enumerate(zip(self.plans, self.amps)):
            _check(_C["sharp_batch_bind"](self.handle, i, _c64(p.c, "state_c"), _c64(p.psi_y, "psi_y"),
                                          _c64(p.psi, "psi"), _c64(p.probe, "probe"),
                                          _f32(a, "amp", (p.K, p.m, p.m)), _f64(p.metrics, "metrics")))
        self.iter = 0

    def step(self, stream=None):
        self.iter += 1
        for p in self.plans:
            p.iter = self.iter
        _check(_C["sharp_batch_step"](self.handle, self.iter, _stream(stream)))

    def tuned_grid(self, m):
        return int(_C["sharp_batch_tuned_grid"](self.handle, int(m)))

    def tuned_shape(self, m):
        """(grid, rows per round trip, stagger ns) chosen for frame size m."""
        g, r, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_C["sharp_batch_tuned_shape"](self.handle, int(m), ctypes.byref(g), ctypes.byref(r), ctypes.byref(st)))
        return g.value, r.value, st.value

    def set_shape(self, m, grid, rows, stagger_ns):
        _check(_C["sharp_batch_set_shape"](self.handle, int(m), int(grid), int(rows), int(stagger_ns)))

    def status(self, stream=None):
        _check(_C["sharp_batch_status"](self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            _check(_C["sharp_batch_destroy"](self.handle))
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class AmpLoss(torch.autograd.Function):
    """L(obj, probe) = sum_i || |F Q(obj, probe)_i| - amp_i ||^2 with the
    hand-written adjoint of the library (frame FFTs recomputed in backward)."""

    @staticmethod
    def forward(ctx, obj, probe, amp, plan_handle):
        loss = torch.zeros(1, dtype=torch.float64, device=obj.device)
        sharp_amp_loss(plan_handle, obj.contiguous(), probe.contiguous(), amp, loss)
        ctx.save_for_backward(obj, probe, amp)
        ctx.plan = plan_handle
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        obj, probe, amp = ctx.saved_tensors
        g_obj = torch.empty_like(obj)
        g_probe = torch.empty_like(probe)
        # torch's gradient of a real loss w.r.t. a complex input is 2 dL/d conj(x)
        scale = 2.0 * float(grad_out.item())
        sharp_amp_loss_backward(ctx.plan, obj.contiguous(), probe.contiguous(), amp, scale, g_obj, g_probe)
        return g_obj, g_probe, None, None


def amp_loss(plan: Plan, obj, probe, amp):
    return AmpLoss.apply(obj, probe, amp, plan.handle)
