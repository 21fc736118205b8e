"""The GPP sum split over ranks by local column (igp).

BerkeleyGW gives each MPI task a slice of the igp columns and the task's kernel sums over
them (paper §II-A); the full sums are the 2*nw complex partial sums added over tasks. Here
every rank holds the whole instance, takes a contiguous column range, runs gpp_sigma on
it, and the partials are gathered and added in rank order, so every rank gets the same
bits whatever the collective's internal order. The exchange is 2 * nw complex numbers per
rank (96 bytes at nw = 3).
"""

from __future__ import annotations

import torch
import torch.distributed as dist

from . import gpp


def column_range(ngpown: int, rank: int, world: int) -> tuple[int, int]:
    """Balanced contiguous range [lo, hi) of the columns owned by ``rank``."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    base, extra = divmod(ngpown, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def restrict_columns(dp: gpp.DeviceProblem, lo: int, hi: int) -> gpp.DeviceProblem:
    """The same instance restricted to local columns [lo, hi) (views, no copies)."""
    return gpp.DeviceProblem(dp.number_bands, dp.nvband, dp.ncouls, hi - lo, dp.nw, dp.aqsmtemp,
                             dp.aqsntemp, dp.I_eps_array[lo:hi], dp.wtilde_array[lo:hi], dp.vcoul,
                             dp.inv_igp_index[lo:hi], dp.indinv, dp.wx_array, dp.aqsntemp_c64)


def reduce_outputs(ach: torch.Tensor, asx: torch.Tensor, group=None):
    """Sum per-rank (achtemp, asxtemp) in rank order on every rank (deterministic). With a
    gloo group the 2 * nw values go through host memory (gloo's collectives are host-side);
    the result comes back on the outputs' device."""
    world = dist.get_world_size(group)
    mine = torch.cat([torch.view_as_real(ach), torch.view_as_real(asx)]).reshape(-1)
    dev = mine.device
    if dist.get_backend(group) == "gloo":
        mine = mine.cpu()
    bufs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    tot = bufs[0].clone()
    for b in bufs[1:]:
        tot += b
    tot = torch.view_as_complex(tot.reshape(-1, 2)).to(dev)
    nw = ach.numel()
    return tot[:nw].clone(), tot[nw:].clone()


def sigma_columns(dp: gpp.DeviceProblem, group=None, **opts):
    """gpp_sigma over this rank's column range, summed over the ranks of ``group``."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    lo, hi = column_range(dp.ngpown, rank, world)
    ach, asx = gpp.sigma(restrict_columns(dp, lo, hi), **opts)
    return reduce_outputs(ach, asx, group)
