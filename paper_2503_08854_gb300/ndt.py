"""ctypes binding of the C ABI in ``include/ndt.h`` (argument marshalling only).

Every function has the name of its C entry point without the ``ndt_``
prefix and forwards raw pointers: torch tensors (CUDA or CPU) and numpy
arrays are accepted and passed as device or host addresses; the library
decides whether to copy.  All computation runs in ``libndt.so``; there is no
fallback: if the library is missing this module raises on import.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libndt.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; "
                      f"g.build()'` (needs nvcc) before using the CUDA path")

_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE, ENOCONV = range(7)
PLANE_F32, PLANE_BF16, PLANE_F16 = 0, 1, 2
LAUNCH_PLAIN, LAUNCH_PERSISTENT = 0, 1
_PLANE_NAMES = {"f32": PLANE_F32, "bf16": PLANE_BF16, "f16": PLANE_F16}


class Exposure(C.Structure):
    _fields_ = [("mjd", C.c_double), ("obs_xyz", C.c_double * 3), ("crval", C.c_double * 2),
                ("crpix", C.c_double * 2), ("cd", C.c_double * 4), ("psf_sigma_px", C.c_float),
                ("variance", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("samples", C.c_int64),
                ("valid_samples", C.c_int64), ("kepler_failures", C.c_int64),
                ("last_stack_ms", C.c_float), ("last_planes_ms", C.c_float),
                ("last_topk_ms", C.c_float), ("orbit_tile", C.c_int32), ("exp_tile", C.c_int32),
                ("launch_mode", C.c_int32), ("plane_dtype", C.c_int32),
                ("offchip_skipped", C.c_int64), ("block_skipped", C.c_int64),
                ("noise_bytes_read", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


assert C.sizeof(Exposure) == 112

_vp, _i32, _i64, _f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_lib.ndt_create.argtypes = [C.POINTER(_vp), C.c_int, _vp]
_lib.ndt_destroy.argtypes = [_vp]
_lib.ndt_destroy.restype = None
_lib.ndt_last_error.argtypes = [_vp]
_lib.ndt_last_error.restype = C.c_char_p
_lib.ndt_set_constants.argtypes = [_vp, _f64, _f64, _f64]
_lib.ndt_load_exposures.argtypes = [_vp, C.POINTER(Exposure), _i32, C.POINTER(_vp), C.POINTER(_vp), _i32]
_lib.ndt_stack_orbits.argtypes = [_vp, _vp, _f64, _i64, _vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp]
_lib.ndt_topk_candidates.argtypes = [_vp, _i64, _vp, _vp, C.POINTER(_i64)]
_lib.ndt_predict_positions.argtypes = [_vp, _vp, _f64, _i64, _vp]
_lib.ndt_get_planes.argtypes = [_vp, _i32, _vp, _vp]
_lib.ndt_set_launch.argtypes = [_vp, _i32, _i32, _i32, _i32]
_lib.ndt_set_offchip_test.argtypes = [_vp, _i32]
_lib.ndt_set_filter_broadening.argtypes = [_vp, C.c_float]
_lib.ndt_selftest_wait_timeout.argtypes = [_vp]
_lib.ndt_trim_candidates.argtypes = [_vp, _vp, _f64, _i64, _vp, _i64, C.c_float, _i32, _i32, _vp, _vp]
_lib.ndt_noise_mad.argtypes = [_vp, C.POINTER(_vp), C.POINTER(_i64), _i32, _i32, _vp, _vp, _vp]
_lib.ndt_autotune.argtypes = [_vp, _vp, _f64, _i64, _vp, _vp, _vp, _i32, _vp]
_lib.ndt_get_stats.argtypes = [_vp, C.POINTER(Stats)]
_lib.ndt_stamps.argtypes = [_vp, _vp, _f64, _i64, _vp, _i64, _vp, _vp]
_lib.ndt_cnn_param_count.argtypes = []
_lib.ndt_cnn_param_count.restype = _i64
_lib.ndt_cnn_forward.argtypes = [_vp, _vp, _vp, _i64, _vp]
_lib.ndt_cnn_loss_grad.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]
_lib.ndt_cnn_adam_step.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _i32, C.c_float, C.c_float,
                                   C.c_float, C.c_float]
_lib.ndt_vet.argtypes = [_vp, _vp, _vp, _f64, _i64, _vp, _i64, _vp]
_lib.ndt_synchronize.argtypes = [_vp]
_lib.ndt_topk_noalloc.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp]
_lib.ndt_dedup_candidates.argtypes = [_vp, _vp, _f64, _i64, _vp, _i64, C.c_float, _i32, _f64, _f64, _vp,
                                      C.POINTER(_i64)]
_lib.ndt_set_block_test.argtypes = [_vp, _i32]
_lib.ndt_set_fp64_geometry.argtypes = [_vp, _i32]
_lib.ndt_set_df_state.argtypes = [_vp, _i32]
_lib.ndt_set_footprint_sort.argtypes = [_vp, _i32]
_lib.ndt_count_candidates.argtypes = [_vp, C.c_float, C.POINTER(_i64)]
_lib.ndt_measure_fp64_rate.argtypes = [C.c_int, _i32, C.POINTER(_f64), C.POINTER(_f64)]


class NdtError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"ndt status {status}: {message}")
        self.status = status


def _ptr(x):
    """Address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array arguments must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check(ctx, status):
    if status != OK:
        raise NdtError(status, _lib.ndt_last_error(ctx).decode())


def create(device=0, stream=None):
    """ndt_create.  ``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    h = _vp()
    raw = getattr(stream, "cuda_stream", stream)
    st = _lib.ndt_create(C.byref(h), int(device), raw)
    if st != OK:
        raise NdtError(st, _lib.ndt_last_error(None).decode())
    return h


def destroy(ctx):
    _lib.ndt_destroy(ctx)


def last_error(ctx):
    return _lib.ndt_last_error(ctx).decode()


def set_constants(ctx, gm, c_light, obliquity_rad):
    _check(ctx, _lib.ndt_set_constants(ctx, gm, c_light, obliquity_rad))


def exposure_table(ex):
    """Marshal a ``synth.Exposures`` table into an array of ndt_exposure."""
    n = len(ex.mjd)
    arr = (Exposure * n)()
    cd = np.asarray(ex.cd, dtype=np.float64).reshape(n, 4)
    for j in range(n):
        e = arr[j]
        e.mjd = float(ex.mjd[j])
        e.obs_xyz[:] = [float(v) for v in ex.obs[j]]
        e.crval[:] = [float(v) for v in ex.crval[j]]
        e.crpix[:] = [float(v) for v in ex.crpix[j]]
        e.cd[:] = [float(v) for v in cd[j]]
        e.psf_sigma_px = float(ex.sigma[j])
        e.variance = float(ex.var[j])
        e.width = int(ex.width[j])
        e.height = int(ex.height[j])
    return arr


def load_exposures(ctx, ex, images, variances=None, plane_dtype="f32"):
    """``images``: a sequence of per-exposure buffers or one (n, H, W) buffer."""
    table = exposure_table(ex)
    n = len(table)
    if hasattr(images, "shape") and len(images.shape) == 3:
        images = [images[j] for j in range(n)]
    ptrs = (_vp * n)(*[_ptr(im) for im in images])
    vptrs = None
    if variances is not None:
        if hasattr(variances, "shape") and len(variances.shape) == 3:
            variances = [variances[j] for j in range(n)]
        vptrs = (_vp * n)(*[_ptr(v) for v in variances])
    dt = _PLANE_NAMES.get(plane_dtype, plane_dtype)
    _check(ctx, _lib.ndt_load_exposures(ctx, table, n, ptrs, vptrs, int(dt)))


def stack_orbits(ctx, states_soa, t0, n_orbits, families=None, min_obs=1, psi_sum=None,
                 phi_sum=None, nobs=None, snr=None):
    """``states_soa``: 6 x n_orbits FP64 buffer (x, y, z, vx, vy, vz rows).
    ``families``: (fam_orbit_off int64, fam_exp_off int64, fam_exp_idx int32) or None."""
    if families is None:
        fo = fe = fi = None
        nf = 0
    else:
        fo, fe, fi = families
        nf = len(fo) - 1
    _check(ctx, _lib.ndt_stack_orbits(ctx, _ptr(states_soa), float(t0), int(n_orbits), _ptr(fo),
                                      _ptr(fe), _ptr(fi), nf, int(min_obs), _ptr(psi_sum),
                                      _ptr(phi_sum), _ptr(nobs), _ptr(snr)))


def topk_candidates(ctx, k, idx_out=None, snr_out=None):
    got = _i64(0)
    _check(ctx, _lib.ndt_topk_candidates(ctx, int(k), _ptr(idx_out), _ptr(snr_out), C.byref(got)))
    return got.value


def predict_positions(ctx, states_soa, t0, n_orbits, xy_out):
    _check(ctx, _lib.ndt_predict_positions(ctx, _ptr(states_soa), float(t0), int(n_orbits),
                                           _ptr(xy_out)))


def get_planes(ctx, j, psi_out=None, phi_out=None):
    _check(ctx, _lib.ndt_get_planes(ctx, int(j), _ptr(psi_out), _ptr(phi_out)))


def set_launch(ctx, mode, orbit_tile=64, exp_tile=16, use_graph=False):
    _check(ctx, _lib.ndt_set_launch(ctx, int(mode), int(orbit_tile), int(exp_tile), int(bool(use_graph))))


def set_filter_broadening(ctx, sigma_px):
    """Matched filter of the next load_exposures broadened by a Gaussian of
    sigma_px (0: the plain filter)."""
    _check(ctx, _lib.ndt_set_filter_broadening(ctx, float(sigma_px)))


def set_offchip_test(ctx, enabled):
    _check(ctx, _lib.ndt_set_offchip_test(ctx, int(bool(enabled))))


def autotune(ctx, states_soa, t0, n_orbits, families=None, times_ms=None):
    if families is None:
        fo = fe = fi = None
        nf = 0
    else:
        fo, fe, fi = families
        nf = len(fo) - 1
    _check(ctx, _lib.ndt_autotune(ctx, _ptr(states_soa), float(t0), int(n_orbits), _ptr(fo),
                                  _ptr(fe), _ptr(fi), nf, _ptr(times_ms)))


def get_stats(ctx):
    s = Stats()
    _check(ctx, _lib.ndt_get_stats(ctx, C.byref(s)))
    return s.as_dict()


def synchronize(ctx):
    _check(ctx, _lib.ndt_synchronize(ctx))


def stamps(ctx, states_soa, t0, n_orbits, cand_idx, stamps_f32=None, stamps_bf16=None):
    """Stacked stamps [n_cand][2][21][21] of candidates (indices into the batch)."""
    _check(ctx, _lib.ndt_stamps(ctx, _ptr(states_soa), float(t0), int(n_orbits), _ptr(cand_idx),
                                int(len(cand_idx)), _ptr(stamps_f32), _ptr(stamps_bf16)))


def cnn_param_count():
    return int(_lib.ndt_cnn_param_count())


def cnn_forward(ctx, params, stamps_bf16, n, logits):
    _check(ctx, _lib.ndt_cnn_forward(ctx, _ptr(params), _ptr(stamps_bf16), int(n), _ptr(logits)))


def cnn_loss_grad(ctx, params, stamps_bf16, labels, n, grad, logits=None):
    """Mean BCE loss (returned) and its gradient (written to ``grad``)."""
    loss = np.zeros(1, np.float32)
    _check(ctx, _lib.ndt_cnn_loss_grad(ctx, _ptr(params), _ptr(stamps_bf16), _ptr(labels), int(n),
                                       _ptr(grad), _ptr(loss), _ptr(logits)))
    return float(loss[0])


def cnn_adam_step(ctx, params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(ctx, _lib.ndt_cnn_adam_step(ctx, _ptr(params), _ptr(grad), _ptr(m), _ptr(v),
                                       int(params.numel() if hasattr(params, "numel") else len(params)),
                                       int(step), lr, beta1, beta2, eps))


def vet(ctx, params, states_soa, t0, n_orbits, cand_idx, scores):
    """Stamps of the candidates scored by the network (sigmoid outputs)."""
    _check(ctx, _lib.ndt_vet(ctx, _ptr(params), _ptr(states_soa), float(t0), int(n_orbits),
                             _ptr(cand_idx), int(len(cand_idx)), _ptr(scores)))


def selftest_wait_timeout(ctx):
    """Status of ndt_selftest_wait_timeout (ETIMEOUT when the bounded waits work)."""
    return _lib.ndt_selftest_wait_timeout(ctx)


def noise_mad(ctx, images, max_rounds=10):
    """Iterative-MAD noise estimate of each image (ndt_noise_mad).  ``images``:
    a sequence of FP32 numpy arrays or torch tensors (host or device).
    Returns numpy arrays (median, sigma, rounds)."""
    n = len(images)
    ptrs = (_vp * max(n, 1))(*[_ptr(x) for x in images])
    npx = (_i64 * max(n, 1))(*[int(x.numel() if hasattr(x, "numel") else x.size) for x in images])
    med = np.zeros(n, np.float32)
    sig = np.zeros(n, np.float32)
    rnd = np.zeros(n, np.int32)
    _check(ctx, _lib.ndt_noise_mad(ctx, ptrs, npx, n, int(max_rounds), _ptr(med), _ptr(sig), _ptr(rnd)))
    return med, sig, rnd


def trim_candidates(ctx, states_soa, t0, n_orbits, cand_idx, nu_out, nkept_out=None, kappa=3.0,
                    max_iter=10, min_obs=1):
    """Outlier-trimmed stacked SNR of the candidates (sigma clipping of their
    intersections, see ndt_trim_candidates)."""
    _check(ctx, _lib.ndt_trim_candidates(ctx, _ptr(states_soa), float(t0), int(n_orbits), _ptr(cand_idx),
                                         int(len(cand_idx)), float(kappa), int(max_iter), int(min_obs),
                                         _ptr(nu_out), _ptr(nkept_out)))


def topk_noalloc(snr, n, k, idx_out=None, snr_out=None, stream=None):
    """ndt_topk_noalloc: top-k of a device array with the library's fixed
    scratch (no device allocation); device pointers only, asynchronous on
    ``stream`` (a torch.cuda.Stream, a raw cudaStream_t, or None)."""
    raw = getattr(stream, "cuda_stream", stream)
    st = _lib.ndt_topk_noalloc(_ptr(snr), int(n), int(k), _ptr(idx_out), _ptr(snr_out), raw)
    if st != OK:
        raise NdtError(st, "ndt_topk_noalloc rejected the call (sizes, or non-device pointers)")


def set_fp64_geometry(ctx, enabled=True):
    """ndt_set_fp64_geometry: FP64 light time and TAN projection in the plain form."""
    _check(ctx, _lib.ndt_set_fp64_geometry(ctx, 1 if enabled else 0))


def set_df_state(ctx, enabled=True):
    """ndt_set_df_state: the two-body state in double-float (FP32 pairs, the
    default) or, with enabled=False, in FP64, in both stack forms and
    predict_positions."""
    _check(ctx, _lib.ndt_set_df_state(ctx, 1 if enabled else 0))


def set_footprint_sort(ctx, enabled=True):
    """ndt_set_footprint_sort: stack_orbits without families walks the orbits
    in sky-footprint order (results in the caller's order)."""
    _check(ctx, _lib.ndt_set_footprint_sort(ctx, 1 if enabled else 0))


def set_block_test(ctx, enabled=True):
    """ndt_set_block_test: the persistent form's per-warp cone test of each
    staged exposure block."""
    _check(ctx, _lib.ndt_set_block_test(ctx, 1 if enabled else 0))


def count_candidates(ctx, min_snr):
    """ndt_count_candidates: orbits of the last stack with nu >= min_snr."""
    c = C.c_int64()
    _check(ctx, _lib.ndt_count_candidates(ctx, float(min_snr), C.byref(c)))
    return c.value


def dedup_candidates(ctx, states_soa, t0, n_orbits, cand_idx, n_cand, keep_idx, radius_px=4.0, n_ref=3,
                     window=None):
    """ndt_dedup_candidates: keep_idx[:returned] = the candidates of cand_idx
    (rank order) with no better-ranked candidate within radius_px at every
    reference exposure (spread over the exposures with epochs in ``window``
    = (t_lo, t_hi), or over all of them); returns that number."""
    t_lo, t_hi = (1.0, 0.0) if window is None else (float(window[0]), float(window[1]))
    nk = C.c_int64()
    _check(ctx, _lib.ndt_dedup_candidates(ctx, _ptr(states_soa), float(t0), int(n_orbits), _ptr(cand_idx),
                                          int(n_cand), float(radius_px), int(n_ref), t_lo, t_hi,
                                          _ptr(keep_idx), C.byref(nk)))
    return nk.value


def measure_fp64_rate(device, op="dfma"):
    """ndt_measure_fp64_rate: FP64 thread-instructions per second the GPU
    sustains for one instruction kind ("dfma", "dmul" or "dadd")."""
    code = {"dfma": 0, "dmul": 1, "dadd": 2}[op]
    rate, sec = C.c_double(), C.c_double()
    st = _lib.ndt_measure_fp64_rate(int(device), code, C.byref(rate), C.byref(sec))
    if st != OK:
        raise NdtError(st, "ndt_measure_fp64_rate failed")
    return rate.value


def exported_symbols():
    """Names of the C entry points this binding uses (all must be exported)."""
    return ["ndt_create", "ndt_destroy", "ndt_last_error", "ndt_set_constants",
            "ndt_load_exposures", "ndt_stack_orbits", "ndt_topk_candidates",
            "ndt_predict_positions", "ndt_get_planes", "ndt_set_launch", "ndt_set_offchip_test",
            "ndt_set_filter_broadening",
            "ndt_autotune",
            "ndt_get_stats", "ndt_synchronize", "ndt_stamps", "ndt_cnn_param_count",
            "ndt_cnn_forward", "ndt_cnn_loss_grad", "ndt_cnn_adam_step", "ndt_vet",
            "ndt_trim_candidates", "ndt_noise_mad", "ndt_selftest_wait_timeout", "ndt_topk_noalloc",
            "ndt_measure_fp64_rate", "ndt_dedup_candidates", "ndt_count_candidates",
            "ndt_set_block_test", "ndt_set_fp64_geometry", "ndt_set_df_state", "ndt_set_footprint_sort"]
