"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the oracle under the tolerances of the method.

Tolerances (written here once, used by every parity test):
  pixel positions  |dx|, |dy| <= 1e-3 px
  stacked SNR      |nu_gpu - nu_oracle| <= 1e-5 * max(1, |nu_oracle|)
                   (nu is a ratio of a zero-mean sum: its noise sigma is 1,
                   so the relative bound is taken against max(1, |nu|))
  Psi              |dPsi| <= 1e-5 * max(sqrt(Phi), |Psi|)   (same scale as nu)
  Phi              relative 1e-5
  n_obs            exact
Samples that the oracle flags as within 1e-6 px of a pixel edge are checked
against the oracle's bracket over both neighbouring pixels instead.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08854_gb300 import ndt

POS_TOL = 1e-3
NU_TOL = 1e-5


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch.device("cuda:0")


class Gpu:
    """A context on a dedicated stream, with helpers returning numpy arrays."""

    def __init__(self):
        self.dev = require_gpu()
        self.stream = torch.cuda.Stream(device=self.dev)
        self.ctx = ndt.create(0, self.stream)

    def close(self):
        if self.ctx is not None:
            ndt.destroy(self.ctx)
            self.ctx = None

    def load(self, ex, imgs, plane="f32", variances=None, host=False):
        if host:
            ndt.load_exposures(self.ctx, ex, np.ascontiguousarray(imgs, np.float32),
                               variances=variances, plane_dtype=plane)
        else:
            d = torch.from_numpy(np.ascontiguousarray(imgs, np.float32)).to(self.dev)
            v = None if variances is None else torch.from_numpy(
                np.ascontiguousarray(variances, np.float32)).to(self.dev)
            torch.cuda.synchronize()
            ndt.load_exposures(self.ctx, ex, d, variances=v, plane_dtype=plane)

    def soa(self, states, host=False):
        a = np.ascontiguousarray(np.asarray(states, np.float64).reshape(-1, 6).T)
        if host:
            return a
        t = torch.from_numpy(a).to(self.dev)
        torch.cuda.synchronize()
        return t

    def stack(self, states, t0, families=None, min_obs=1, host=False):
        n = len(states)
        st = self.soa(states, host)
        if host:
            out = dict(psi=np.zeros(n, np.float32), phi=np.zeros(n, np.float32),
                       nobs=np.zeros(n, np.int32), snr=np.zeros(n, np.float32))
            fam = None if families is None else tuple(np.ascontiguousarray(x) for x in families)
            ndt.stack_orbits(self.ctx, st, t0, n, families=fam, min_obs=min_obs,
                             psi_sum=out["psi"], phi_sum=out["phi"], nobs=out["nobs"],
                             snr=out["snr"])
            return out
        out = dict(psi=torch.empty(n, device=self.dev), phi=torch.empty(n, device=self.dev),
                   nobs=torch.empty(n, dtype=torch.int32, device=self.dev),
                   snr=torch.empty(n, device=self.dev))
        fam = None
        if families is not None:
            fam = tuple(torch.from_numpy(np.ascontiguousarray(x)).to(self.dev) for x in families)
            torch.cuda.synchronize()
        ndt.stack_orbits(self.ctx, st, t0, n, families=fam, min_obs=min_obs, psi_sum=out["psi"],
                         phi_sum=out["phi"], nobs=out["nobs"], snr=out["snr"])
        ndt.synchronize(self.ctx)
        return {k: v.cpu().numpy() for k, v in out.items()}

    def topk(self, k, host=False):
        if host:
            idx = np.zeros(k, np.int64)
            val = np.zeros(k, np.float32)
            got = ndt.topk_candidates(self.ctx, k, idx, val)
            return idx[:got], val[:got]
        idx = torch.empty(k, dtype=torch.int64, device=self.dev)
        val = torch.empty(k, device=self.dev)
        got = ndt.topk_candidates(self.ctx, k, idx, val)
        return idx[:got].cpu().numpy(), val[:got].cpu().numpy()

    def predict(self, states, t0, n_exp):
        n = len(states)
        xy = torch.empty(n * n_exp * 2, dtype=torch.float64, device=self.dev)
        ndt.predict_positions(self.ctx, self.soa(states), t0, n, xy)
        return xy.cpu().numpy().reshape(n, n_exp, 2)

    def planes(self, j, H, W):
        psi = torch.empty(H * W, device=self.dev)
        phi = torch.empty(H * W, device=self.dev)
        ndt.get_planes(self.ctx, j, psi, phi)
        return psi.cpu().numpy().reshape(H, W), phi.cpu().numpy().reshape(H, W)

    def stats(self):
        return ndt.get_stats(self.ctx)


def check_stack(gpu, ref, min_obs=1):
    """Element-wise parity of one stack against the oracle; returns a report."""
    Psi, Phi, nobs = ref["Psi"], ref["Phi"], ref["nobs"]
    amb = ref["n_amb"] > 0
    clean = ~amb
    g_psi = gpu["psi"].astype(np.float64)
    g_phi = gpu["phi"].astype(np.float64)
    assert np.array_equal(gpu["nobs"][clean], nobs[clean]), \
        f"n_obs mismatch at {np.flatnonzero(gpu['nobs'][clean] != nobs[clean])[:10]}"
    scale = np.maximum(np.sqrt(np.maximum(Phi, 0)), np.abs(Psi))
    d_psi = np.abs(g_psi - Psi)
    assert np.all(d_psi[clean] <= NU_TOL * np.maximum(scale[clean], 1e-30) + 1e-30), \
        f"Psi mismatch: worst {np.max(d_psi[clean] / np.maximum(scale[clean], 1e-30)):.3g}"
    d_phi = np.abs(g_phi - Phi)
    assert np.all(d_phi[clean] <= NU_TOL * np.abs(Phi[clean]) + 1e-30), "Phi mismatch"
    nu = O.snr(Psi, Phi, nobs, min_obs)
    g_nu = gpu["snr"].astype(np.float64)
    fin = clean & np.isfinite(nu)
    assert np.array_equal(np.isfinite(g_nu[clean]), np.isfinite(nu[clean])), "-inf pattern differs"
    err = np.abs(g_nu[fin] - nu[fin]) / np.maximum(1.0, np.abs(nu[fin]))
    assert err.size == 0 or err.max() <= NU_TOL, f"SNR mismatch: worst {err.max():.3g}"
    # ambiguous orbits: inside the oracle's bracket
    if amb.any():
        tol_a = NU_TOL * np.maximum(scale[amb], 1e-12) + 1e-6
        assert np.all(g_psi[amb] >= ref["psi_lo"][amb] - tol_a)
        assert np.all(g_psi[amb] <= ref["psi_hi"][amb] + tol_a)
        assert np.all(gpu["nobs"][amb] >= ref["n_lo"][amb])
        assert np.all(gpu["nobs"][amb] <= ref["n_hi"][amb])
    return dict(max_rel_snr_err=float(err.max()) if err.size else 0.0,
                n_ambiguous=int(amb.sum()), n_finite=int(fin.sum()))


def check_topk(g_idx, g_val, ref_nu, amb, k):
    """The GPU ranking equals the oracle's, except where two oracle values at
    the same rank lie within the SNR tolerance (a near-tie) or an orbit with
    an edge-ambiguous sample is involved."""
    o_idx, o_val = O.topk(ref_nu, k)
    assert len(g_idx) == len(o_idx)
    assert len(set(g_idx.tolist())) == len(g_idx), "duplicate index in GPU top-k"
    swaps = 0
    for i in range(len(o_idx)):
        if g_idx[i] == o_idx[i]:
            continue
        a, b = ref_nu[g_idx[i]], ref_nu[o_idx[i]]
        near = (a == b) or abs(a - b) <= 2 * NU_TOL * max(1.0, abs(b))
        assert near or amb[g_idx[i]] or amb[o_idx[i]], \
            f"rank {i}: GPU {g_idx[i]} (nu {a}) vs oracle {o_idx[i]} (nu {b})"
        swaps += 1
    fin = np.isfinite(o_val)
    assert np.all(np.abs(g_val[fin] - o_val[fin]) <= NU_TOL * np.maximum(1, np.abs(o_val[fin])) * 2)
    return swaps
