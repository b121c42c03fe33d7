"""Coarse-to-fine orbit search (paper sec. 5.2.4: smoothing the images with a
Gaussian wider than the PSF allows sparser sampling of orbits while still
gaining signal from objects on adjacent orbits).

Over a regular grid of candidate orbits (any number of dimensions), the
coarse pass stacks every ``stride``-th node along each axis against planes
whose matched filter is broadened by ``broaden_px``; the fine pass reloads
the plain planes and stacks, at full resolution, the nodes within
``radius`` of the ``k_coarse`` best coarse nodes.  Every stack and ranking
runs in the library; this module only chooses grid indices."""
import numpy as np

from . import ndt


def _stack_rank(ctx, states_rows, t0, k, device):
    import torch
    n = len(states_rows)
    st = torch.from_numpy(np.ascontiguousarray(np.asarray(states_rows, np.float64).T)).to(device)
    snr = torch.empty(n, device=device)
    torch.cuda.synchronize(device)
    ndt.stack_orbits(ctx, st, 0.0 + t0, n, snr=snr)
    k = min(k, n)
    idx = torch.empty(k, dtype=torch.int64, device=device)
    val = torch.empty(k, device=device)
    got = ndt.topk_candidates(ctx, k, idx, val)
    return idx[:got].cpu().numpy(), val[:got].cpu().numpy(), snr.cpu().numpy()


def coarse_to_fine(ctx, ex, images, grid_states, t0, *, stride=4, broaden_px=2.0, k_coarse=4,
                   radius=None, k=10, device=None):
    """``grid_states``: (n_1, ..., n_d, 6) orbit states on a regular grid.
    Returns a dict: ``best`` (grid multi-indices of the k best fine nodes),
    ``nu`` (their SNR), ``coarse_best`` (multi-indices of the coarse winners),
    ``coarse_nu``, ``evaluated`` (orbits stacked in both passes) and
    ``dense`` (the grid size)."""
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    grid_states = np.asarray(grid_states, np.float64)
    shape = grid_states.shape[:-1]
    radius = stride if radius is None else radius
    # coarse pass
    coarse_axes = [np.arange(0, n, stride) for n in shape]
    cmesh = np.stack(np.meshgrid(*coarse_axes, indexing="ij"), -1).reshape(-1, len(shape))
    ndt.set_filter_broadening(ctx, broaden_px)
    try:
        ndt.load_exposures(ctx, ex, images)
    finally:
        ndt.set_filter_broadening(ctx, 0.0)
    c_idx, c_val, _ = _stack_rank(ctx, grid_states[tuple(cmesh.T)], t0, k_coarse, device)
    winners = cmesh[c_idx]
    # fine pass around the winners
    ndt.load_exposures(ctx, ex, images)
    cells = set()
    span = np.arange(-radius, radius + 1)
    for w in winners:
        local = np.stack(np.meshgrid(*[w[a] + span for a in range(len(shape))], indexing="ij"),
                         -1).reshape(-1, len(shape))
        ok = np.all((local >= 0) & (local < np.asarray(shape)), axis=1)
        cells.update(map(tuple, local[ok]))
    fine = np.array(sorted(cells), dtype=np.int64)
    f_idx, f_val, _ = _stack_rank(ctx, grid_states[tuple(fine.T)], t0, k, device)
    return {"best": fine[f_idx], "nu": f_val, "coarse_best": winners, "coarse_nu": c_val,
            "evaluated": len(cmesh) + len(fine), "dense": int(np.prod(shape))}
