"""ctypes front end of the FP64 C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function is a
thin call into the C reference; the arithmetic lives in ``oracle.c`` and
each C function cites the part of arXiv 2503.08854 it follows.
"""
import ctypes as C
import os

import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.orc_gm_sun.restype = C.c_double
        L.orc_c_light.restype = C.c_double
        L.orc_obliquity.restype = C.c_double
        L.orc_kepler_uv.argtypes = [dp, dp, C.c_double, C.c_double, dp, dp, dp]
        L.orc_kepler_uv.restype = C.c_int
        L.orc_apparent.argtypes = [dp, C.c_double, C.c_double, dp, C.c_double, C.c_double, dp, dp]
        L.orc_apparent.restype = C.c_int
        L.orc_project.argtypes = [dp, C.c_double, dp, dp, dp, dp, dp, dp]
        L.orc_project.restype = C.c_int
        L.orc_psf_kernel.argtypes = [C.c_double, dp, C.c_int]
        L.orc_psf_kernel.restype = C.c_int
        L.orc_planes.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_double,
                                 dp, dp]
        L.orc_planes.restype = C.c_int
        L.orc_predict.argtypes = [dp, C.c_int64, C.c_double, C.c_void_p, C.c_double, C.c_double,
                                  C.c_double, dp, C.c_int]
        L.orc_predict.restype = C.c_int
        L.orc_stack.argtypes = [dp, C.c_int64, C.c_double, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_double, C.c_double, C.c_double, C.c_double,
                                dp, dp, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.orc_stack.restype = C.c_int
        L.orc_snr.argtypes = [dp, dp, C.c_void_p, C.c_int64, C.c_int32, dp]
        L.orc_topk.argtypes = [dp, C.c_int64, C.c_int64, C.c_void_p, dp]
        L.orc_topk.restype = C.c_int
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gm_sun():
    return lib().orc_gm_sun()


def c_light():
    return lib().orc_c_light()


def obliquity():
    return lib().orc_obliquity()


def max_threads():
    return lib().orc_max_threads()


def kepler(r0, v0, dt, mu=None):
    """Universal-variable two-body step.  Returns (r, v, (f, g, fdot, gdot), iterations)."""
    mu = gm_sun() if mu is None else mu
    r0, v0 = _f64(r0), _f64(v0)
    r, v, fg = np.zeros(3), np.zeros(3), np.zeros(4)
    it = lib().orc_kepler_uv(_d(r0), _d(v0), float(dt), float(mu), _d(r), _d(v), _d(fg))
    if it < 0:
        raise RuntimeError("oracle Kepler solve did not converge")
    return r, v, fg, it


def apparent(state, t0, t_obs, obs, mu=None, c=None):
    """Light-time corrected topocentric vector rho and light time tau."""
    mu = gm_sun() if mu is None else mu
    c = c_light() if c is None else c
    state, obs = _f64(state), _f64(obs)
    rho, tau = np.zeros(3), np.zeros(1)
    if lib().orc_apparent(_d(state), float(t0), float(t_obs), _d(obs), float(mu), float(c),
                          _d(rho), _d(tau)) != 0:
        raise RuntimeError("oracle light-time solve failed")
    return rho, float(tau[0])


def project(rho, crval, crpix, cd, eps=None):
    """TAN projection of a topocentric ecliptic vector.  Returns (valid, x, y, ra, dec)."""
    eps = obliquity() if eps is None else eps
    rho = _f64(rho)
    crval, crpix, cd = _f64(crval), _f64(crpix), _f64(np.asarray(cd).reshape(4))
    x, y, rd = np.zeros(1), np.zeros(1), np.zeros(2)
    ok = lib().orc_project(_d(rho), float(eps), _d(crval), _d(crpix), _d(cd), _d(x), _d(y), _d(rd))
    return bool(ok), float(x[0]), float(y[0]), float(rd[0]), float(rd[1])


def psf_kernel(sigma):
    R = int(np.ceil(4.0 * sigma))
    n = 2 * R + 1
    P = np.zeros(n * n)
    lib().orc_psf_kernel(float(sigma), _d(P), n * n)
    return P.reshape(n, n)


def planes(img, sigma, var=1.0):
    """psi, phi planes (FP64) of one FP32 image; ``var`` a scalar or a FP32 plane."""
    img = np.ascontiguousarray(img, dtype=np.float32)
    H, W = img.shape
    psi, phi = np.zeros((H, W)), np.zeros((H, W))
    if np.isscalar(var):
        vp, vc = None, float(var)
    else:
        var = np.ascontiguousarray(var, dtype=np.float32)
        vp, vc = var.ctypes.data, 1.0
    lib().orc_planes(img.ctypes.data, vp, vc, W, H, float(sigma), _d(psi), _d(phi))
    return psi, phi


class _ExpStruct(C.Structure):
    _fields_ = [("n", C.c_int), ("mjd", C.c_void_p), ("obs", C.c_void_p), ("crval", C.c_void_p),
                ("crpix", C.c_void_p), ("cd", C.c_void_p), ("sigma", C.c_void_p),
                ("var", C.c_void_p), ("width", C.c_void_p), ("height", C.c_void_p)]


def _exp_struct(ex):
    """Marshal an exposure table (``synth.Exposures``) into the C struct."""
    keep = dict(
        mjd=_f64(ex.mjd), obs=_f64(ex.obs), crval=_f64(ex.crval), crpix=_f64(ex.crpix),
        cd=_f64(np.asarray(ex.cd).reshape(-1, 4)), sigma=_f64(ex.sigma), var=_f64(ex.var),
        width=np.ascontiguousarray(ex.width, dtype=np.int32),
        height=np.ascontiguousarray(ex.height, dtype=np.int32))
    s = _ExpStruct(len(keep["mjd"]), *[keep[k].ctypes.data for k in
                                       ("mjd", "obs", "crval", "crpix", "cd", "sigma", "var",
                                        "width", "height")])
    return s, keep


def predict(states, t0, ex, mu=None, c=None, eps=None, nthreads=0):
    """Pixel coordinates [n_o, n_exp, 2] (NaN where cos c <= 0)."""
    mu = gm_sun() if mu is None else mu
    c = c_light() if c is None else c
    eps = obliquity() if eps is None else eps
    states = _f64(states).reshape(-1, 6)
    s, keep = _exp_struct(ex)
    xy = np.zeros((states.shape[0], s.n, 2))
    if lib().orc_predict(_d(states), states.shape[0], float(t0), C.byref(s), float(mu), float(c),
                         float(eps), _d(xy), int(nthreads)) != 0:
        raise RuntimeError("oracle prediction failed")
    return xy


def _ptr_array(arrs, dtype):
    arrs = [np.ascontiguousarray(a, dtype=dtype) for a in arrs]
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return ptrs, arrs


def stack(states, t0, ex, images=None, var_planes=None, planes=None, families=None,
          mu=None, c=None, eps=None, amb_px=1e-6, nthreads=0):
    """Brute-force stack.  ``planes`` = (list of psi, list of phi) FP64 planes, or
    ``images`` (list of FP32 images) to evaluate the planes at the gathered pixel.
    ``families`` = (fam_orb_off int64, fam_exp_off int64, fam_exp_idx int32) or None.
    Returns a dict of per-orbit arrays."""
    mu = gm_sun() if mu is None else mu
    c = c_light() if c is None else c
    eps = obliquity() if eps is None else eps
    states = _f64(states).reshape(-1, 6)
    n_o = states.shape[0]
    s, keep = _exp_struct(ex)
    hold = []
    img_p = var_p = psi_p = phi_p = None
    if planes is not None:
        psi_p, a = _ptr_array(planes[0], np.float64); hold.append(a)
        phi_p, a = _ptr_array(planes[1], np.float64); hold.append(a)
    else:
        img_p, a = _ptr_array(images, np.float32); hold.append(a)
        if var_planes is not None:
            var_p, a = _ptr_array(var_planes, np.float32); hold.append(a)
    if families is not None:
        fo = np.ascontiguousarray(families[0], dtype=np.int64)
        fe = np.ascontiguousarray(families[1], dtype=np.int64)
        fi = np.ascontiguousarray(families[2], dtype=np.int32)
        nf, fo_p, fe_p, fi_p = len(fo) - 1, fo.ctypes.data, fe.ctypes.data, fi.ctypes.data
    else:
        nf, fo_p, fe_p, fi_p = 0, None, None, None
    out = {k: np.zeros(n_o) for k in ("Psi", "Phi", "psi_lo", "psi_hi", "phi_lo", "phi_hi")}
    for k in ("nobs", "n_lo", "n_hi", "n_amb"):
        out[k] = np.zeros(n_o, dtype=np.int32)
    rc = lib().orc_stack(
        _d(states), n_o, float(t0), C.byref(s), img_p, var_p, psi_p, phi_p,
        nf, fo_p, fe_p, fi_p, float(mu), float(c), float(eps), float(amb_px),
        _d(out["Psi"]), _d(out["Phi"]), out["nobs"].ctypes.data,
        out["psi_lo"].ctypes.data, out["psi_hi"].ctypes.data,
        out["phi_lo"].ctypes.data, out["phi_hi"].ctypes.data,
        out["n_lo"].ctypes.data, out["n_hi"].ctypes.data, out["n_amb"].ctypes.data, int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle stack failed")
    return out


def snr(Psi, Phi, nobs, min_obs=1):
    Psi, Phi = _f64(Psi), _f64(Phi)
    nobs = np.ascontiguousarray(nobs, dtype=np.int32)
    nu = np.zeros(len(Psi))
    lib().orc_snr(_d(Psi), _d(Phi), nobs.ctypes.data, len(Psi), int(min_obs), _d(nu))
    return nu


def topk(nu, k):
    nu = _f64(nu)
    idx = np.zeros(max(k, 1), dtype=np.int64)
    val = np.zeros(max(k, 1))
    got = lib().orc_topk(_d(nu), len(nu), int(k), idx.ctypes.data, _d(val))
    return idx[:got], val[:got]
