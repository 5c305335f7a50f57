"""ctypes binding of the C ABI in include/fftenkf.h: same names, argument marshalling only.

Every function here forwards to the shared library built from csrc/; nothing is
computed in Python.  Import fails loudly if the library is missing.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfftenkf.so")

FFTENKF_OK = 0
FFTENKF_EINVAL = 1
FFTENKF_EUNSUPPORTED = 2
FFTENKF_ECUDA = 3
FFTENKF_ENONFINITE = 4
FFTENKF_ETIMEOUT = 5
FFTENKF_ENOMEM = 6
FFTENKF_F32 = 0
FFTENKF_BF16 = 1


class fftenkf_dims(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nx", ctypes.c_int), ("n_blocks", ctypes.c_int),
                ("n_members", ctypes.c_int), ("storage", ctypes.c_int)]


class FftEnkfError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__("%s: %s (%s)" % (where, fftenkf_status_string(status), message))
        self.status = status


_lib = None

# (name, restype, argtypes)
_SIGNATURES = [
    ("fftenkf_plan_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(fftenkf_dims), ctypes.c_char_p]),
    ("fftenkf_plan_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("fftenkf_workspace_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("fftenkf_spectrum_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("fftenkf_estimate_spectrum", ctypes.c_int, [ctypes.c_void_p] * 5),
    ("fftenkf_analyze", ctypes.c_int, [ctypes.c_void_p] * 8),
    ("fftenkf_analyze_seeded", ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_ulonglong] + [ctypes.c_void_p] * 2),
    ("fftenkf_estimate_spectrum_static", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("fftenkf_static_last_device_status", ctypes.c_int, [ctypes.c_void_p]),
    ("fftenkf_last_device_status", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("fftenkf_set_profiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("fftenkf_pass_times", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("fftenkf_pass_count", ctypes.c_int, []),
    ("fftenkf_set_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("fftenkf_get_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("fftenkf_set_coupled", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("fftenkf_set_expire_first_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("fftenkf_pass_name", ctypes.c_char_p, [ctypes.c_int]),
    ("fftenkf_plan_batched", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(fftenkf_dims)]),
    ("fftenkf_batch_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("fftenkf_batch_workspace_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("fftenkf_analyze_batched", ctypes.c_int, [ctypes.c_void_p] * 7),
    ("fftenkf_batch_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.POINTER(ctypes.c_double)]),
    ("fftenkf_batch_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("fftenkf_batch_last_device_status", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("fftenkf_mlp_param_count", ctypes.c_int, []),
    ("fftenkf_denoiser_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("fftenkf_denoiser_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("fftenkf_denoiser_features", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    ("fftenkf_mlp_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("fftenkf_mlp_gradient", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fftenkf_mlp_adam", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_float, ctypes.c_void_p]),
    ("fftenkf_denoise_spectrum", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    ("fftenkf_sine_plan_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(fftenkf_dims),
                                                ctypes.c_char_p]),
    ("fftenkf_sine_plan_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("fftenkf_sine_spectrum_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("fftenkf_sine_estimate_spectrum", ctypes.c_int, [ctypes.c_void_p] * 4),
    ("fftenkf_sine_analyze", ctypes.c_int, [ctypes.c_void_p] * 6),
    ("fftenkf_sine_last_device_status", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("fftenkf_morph_forward", ctypes.c_int,
     [ctypes.c_void_p] * 3 + [ctypes.c_int] * 5 + [ctypes.c_float, ctypes.c_void_p]),
    ("fftenkf_morph_reference", ctypes.c_int, [ctypes.c_void_p] * 2 + [ctypes.c_int] * 4 + [ctypes.c_void_p]),
    ("fftenkf_morph_inverse", ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int] * 4 + [ctypes.c_void_p]),
    ("fftenkf_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("fftenkf_last_error", ctypes.c_char_p, []),
]


def lib() -> ctypes.CDLL:
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfftenkf.so not built; run `python -m paper_1001_1588_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    """Names of the entry points the binding knows about."""
    return [s[0] for s in _SIGNATURES]


def fftenkf_status_string(status: int) -> str:
    return lib().fftenkf_status_string(status).decode()


def fftenkf_last_error() -> str:
    return lib().fftenkf_last_error().decode()


def check(status: int, where: str) -> None:
    if status != FFTENKF_OK:
        raise FftEnkfError(status, where, fftenkf_last_error())


def _p(x):
    """Pointer argument: None, int address, or an object with data_ptr()."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def fftenkf_plan_create(ny, nx, n_blocks, n_members, storage, observed_mask):
    d = fftenkf_dims(ny, nx, n_blocks, n_members, storage)
    plan = ctypes.c_void_p()
    mask = bytes(int(bool(m)) for m in observed_mask)
    check(lib().fftenkf_plan_create(ctypes.byref(plan), ctypes.byref(d), mask), "fftenkf_plan_create")
    return plan.value


def fftenkf_plan_destroy(plan):
    check(lib().fftenkf_plan_destroy(plan), "fftenkf_plan_destroy")


def fftenkf_workspace_size(plan) -> int:
    n = ctypes.c_size_t()
    check(lib().fftenkf_workspace_size(plan, ctypes.byref(n)), "fftenkf_workspace_size")
    return n.value


def fftenkf_spectrum_size(plan) -> int:
    n = ctypes.c_size_t()
    check(lib().fftenkf_spectrum_size(plan, ctypes.byref(n)), "fftenkf_spectrum_size")
    return n.value


def fftenkf_estimate_spectrum(plan, ensemble, spectrum_out, workspace=None, stream=None):
    check(lib().fftenkf_estimate_spectrum(plan, _p(ensemble), _p(spectrum_out), _p(workspace), stream),
          "fftenkf_estimate_spectrum")


def fftenkf_analyze(plan, ensemble, data, perturbations, rhat, spectrum=None, workspace=None, stream=None):
    check(lib().fftenkf_analyze(plan, _p(ensemble), _p(data), _p(perturbations), _p(rhat), _p(spectrum),
                                _p(workspace), stream), "fftenkf_analyze")


def fftenkf_analyze_seeded(plan, ensemble, data, rhat, seed, spectrum=None, workspace=None, stream=None):
    check(lib().fftenkf_analyze_seeded(plan, _p(ensemble), _p(data), _p(rhat), _p(spectrum), int(seed),
                                       _p(workspace), stream), "fftenkf_analyze_seeded")


def fftenkf_estimate_spectrum_static(ensemble, ny, nx, n_members, storage, spectrum_out, stream=None):
    """Allocation-free single-block estimate (scratch in the library's static device array)."""
    check(lib().fftenkf_estimate_spectrum_static(_p(ensemble), ny, nx, n_members, storage, _p(spectrum_out), stream),
          "fftenkf_estimate_spectrum_static")


def fftenkf_static_last_device_status(stream=None) -> int:
    """Status word of the allocation-free calls on the current device (waits for the stream, clears it)."""
    return lib().fftenkf_static_last_device_status(stream)


def fftenkf_sine_plan_create(ny, nx, n_blocks, n_members, storage, observed_mask):
    d = fftenkf_dims(ny, nx, n_blocks, n_members, storage)
    plan = ctypes.c_void_p()
    mask = bytes(int(bool(m)) for m in observed_mask)
    check(lib().fftenkf_sine_plan_create(ctypes.byref(plan), ctypes.byref(d), mask), "fftenkf_sine_plan_create")
    return plan.value


def fftenkf_sine_plan_destroy(plan):
    check(lib().fftenkf_sine_plan_destroy(plan), "fftenkf_sine_plan_destroy")


def fftenkf_sine_spectrum_size(plan) -> int:
    n = ctypes.c_size_t()
    check(lib().fftenkf_sine_spectrum_size(plan, ctypes.byref(n)), "fftenkf_sine_spectrum_size")
    return n.value


def fftenkf_sine_estimate_spectrum(plan, ensemble, spectrum_out, stream=None):
    check(lib().fftenkf_sine_estimate_spectrum(plan, _p(ensemble), _p(spectrum_out), stream),
          "fftenkf_sine_estimate_spectrum")


def fftenkf_sine_analyze(plan, ensemble, data, perturbations, rhat, stream=None):
    check(lib().fftenkf_sine_analyze(plan, _p(ensemble), _p(data), _p(perturbations), _p(rhat), stream),
          "fftenkf_sine_analyze")


def fftenkf_sine_last_device_status(plan, stream=None) -> int:
    return lib().fftenkf_sine_last_device_status(plan, stream)


def fftenkf_morph_forward(u, u_ref, ext, n_blocks, n_members, ny, nx, n_iter, tol=0.0, stream=None):
    check(lib().fftenkf_morph_forward(_p(u), _p(u_ref), _p(ext), n_blocks, n_members, ny, nx, n_iter, tol, stream),
          "fftenkf_morph_forward")


def fftenkf_morph_reference(ext, ext_ref, n_channels, n_members, ny, nx, stream=None):
    check(lib().fftenkf_morph_reference(_p(ext), _p(ext_ref), n_channels, n_members, ny, nx, stream),
          "fftenkf_morph_reference")


def fftenkf_morph_inverse(ext, u_ref, u_out, n_blocks, n_members, ny, nx, stream=None):
    check(lib().fftenkf_morph_inverse(_p(ext), _p(u_ref), _p(u_out), n_blocks, n_members, ny, nx, stream),
          "fftenkf_morph_inverse")


def fftenkf_last_device_status(plan, stream=None) -> int:
    return lib().fftenkf_last_device_status(plan, stream)


def fftenkf_set_profiling(plan, enable: bool):
    check(lib().fftenkf_set_profiling(plan, int(bool(enable))), "fftenkf_set_profiling")


def fftenkf_pass_count() -> int:
    return lib().fftenkf_pass_count()


def fftenkf_pass_name(i: int) -> str:
    return lib().fftenkf_pass_name(i).decode()


def fftenkf_pass_times(plan):
    """{pass name: (total ms, launches)} since the last read; waits for the events."""
    n = fftenkf_pass_count()
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    check(lib().fftenkf_pass_times(plan, ms, cnt, n), "fftenkf_pass_times")
    return {fftenkf_pass_name(i): (ms[i], cnt[i]) for i in range(n)}


def fftenkf_set_schedule(plan, sched):
    arr = (ctypes.c_int * len(sched))(*[int(x) for x in sched])
    check(lib().fftenkf_set_schedule(plan, arr, len(sched)), "fftenkf_set_schedule")


def fftenkf_set_coupled(plan, coupled):
    check(lib().fftenkf_set_coupled(plan, int(bool(coupled))), "fftenkf_set_coupled")


def fftenkf_set_expire_first_wait(plan, on):
    """Test setting: every CTA of the forward anomaly row pass gives up its first bulk-copy wait."""
    check(lib().fftenkf_set_expire_first_wait(plan, int(bool(on))), "fftenkf_set_expire_first_wait")


def fftenkf_get_schedule(plan):
    n = fftenkf_pass_count()
    arr = (ctypes.c_int * n)()
    check(lib().fftenkf_get_schedule(plan, arr, n), "fftenkf_get_schedule")
    return list(arr)


# ---------------------------------------------------------------- batched
def fftenkf_plan_batched(dims, storage):
    """dims: sequence of (ny, nx, n_members); one observed block each."""
    arr = (fftenkf_dims * len(dims))(*[fftenkf_dims(ny, nx, 1, n, storage) for ny, nx, n in dims])
    b = ctypes.c_void_p()
    check(lib().fftenkf_plan_batched(ctypes.byref(b), len(dims), arr), "fftenkf_plan_batched")
    return b.value


def fftenkf_batch_destroy(b):
    check(lib().fftenkf_batch_destroy(b), "fftenkf_batch_destroy")


def fftenkf_batch_workspace_size(b) -> int:
    n = ctypes.c_size_t()
    check(lib().fftenkf_batch_workspace_size(b, ctypes.byref(n)), "fftenkf_batch_workspace_size")
    return n.value


def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[_p(x) for x in xs])


def fftenkf_analyze_batched(b, ensembles, data, perturbations, rhat, workspace=None, stream=None):
    check(lib().fftenkf_analyze_batched(b, _ptr_array(ensembles), _ptr_array(data), _ptr_array(perturbations),
                                        _ptr_array(rhat), _p(workspace), stream), "fftenkf_analyze_batched")


def fftenkf_batch_autotune(b, workspace=None, stream=None) -> float:
    ms = ctypes.c_double()
    check(lib().fftenkf_batch_autotune(b, _p(workspace), stream, ctypes.byref(ms)), "fftenkf_batch_autotune")
    return ms.value


def fftenkf_batch_schedule(b, n=7):
    bt = (ctypes.c_int * n)()
    sc = (ctypes.c_int * n)()
    check(lib().fftenkf_batch_schedule(b, bt, sc, n), "fftenkf_batch_schedule")
    return list(bt), list(sc)


def fftenkf_batch_last_device_status(b, stream=None) -> int:
    return lib().fftenkf_batch_last_device_status(b, stream)


# ---------------------------------------------------------------- learned spectrum
def fftenkf_mlp_param_count() -> int:
    return lib().fftenkf_mlp_param_count()


def fftenkf_denoiser_create(ny, nx, trained_members=5):
    d = ctypes.c_void_p()
    check(lib().fftenkf_denoiser_create(ctypes.byref(d), ny, nx, trained_members), "fftenkf_denoiser_create")
    return d.value


def fftenkf_denoiser_destroy(d):
    check(lib().fftenkf_denoiser_destroy(d), "fftenkf_denoiser_destroy")


def fftenkf_denoiser_features(d, chat, batch, features, means, stream=None):
    check(lib().fftenkf_denoiser_features(d, _p(chat), batch, _p(features), _p(means), stream),
          "fftenkf_denoiser_features")


def fftenkf_mlp_forward(params, features, batch, out, stream=None):
    check(lib().fftenkf_mlp_forward(_p(params), _p(features), batch, _p(out), stream), "fftenkf_mlp_forward")


def fftenkf_mlp_gradient(params, features, targets, batch, grads, loss, stream=None):
    check(lib().fftenkf_mlp_gradient(_p(params), _p(features), _p(targets), batch, _p(grads), _p(loss), stream),
          "fftenkf_mlp_gradient")


def fftenkf_mlp_adam(params, m, v, grads, step, lr, stream=None):
    check(lib().fftenkf_mlp_adam(_p(params), _p(m), _p(v), _p(grads), step, lr, stream), "fftenkf_mlp_adam")


def fftenkf_denoise_spectrum(d, params, chat_in, chat_out, n_members, stream=None, want_flag=True):
    flag = ctypes.c_int(0)
    check(lib().fftenkf_denoise_spectrum(d, _p(params), _p(chat_in), _p(chat_out), n_members,
                                         ctypes.byref(flag) if want_flag else None, stream),
          "fftenkf_denoise_spectrum")
    return flag.value
