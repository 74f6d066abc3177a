"""Multi-process decomposition of the time-domain method (Sec. 4.2 of the paper).

Two schemes, one process per GPU:
  detector parallelization  every rank holds all trajectories and a contiguous
                            block of pixels; ranks never exchange data during
                            the computation, results are concatenated at the end;
  beam parallelization      every rank holds all pixels and a contiguous block of
                            electrons; records are summed over ranks at the end
                            (superposition is linear), before the spectrum.
Memory per rank follows Eq. (parallel_scheme_function): detector
parallelization needs less whenever N_obs N_Tu >= 4 N_p, which is the usual
case and the default here.
"""
from __future__ import annotations


def balanced_range(n: int, rank: int, world: int):
    """Contiguous [lo, hi) block of n items for `rank` out of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def pixel_shard(n_pix: int, rank: int, world: int):
    """Detector parallelization: this rank's pixel block."""
    return balanced_range(n_pix, rank, world)


def beam_shard(n_e: int, rank: int, world: int):
    """Beam parallelization: this rank's electron block."""
    return balanced_range(n_e, rank, world)


def memory_per_rank(scheme: str, P: int, N_p: int, N_obs: int, N_Tu: int) -> float:
    """Floating-point numbers per process, Sec. 4.2 (M_beam, M_detector)."""
    if scheme == "beam":
        return 12.0 * N_p / P + N_obs * (4.0 * N_p / P + 3.0 * N_Tu)
    if scheme == "detector":
        return 12.0 * N_p + N_obs / P * (4.0 * N_p + 3.0 * N_Tu)
    raise ValueError(scheme)


def preferred_scheme(N_p: int, N_obs: int, N_Tu: int) -> str:
    """Eq. (parallel_scheme_function_2): detector iff N_obs N_Tu >= 4 N_p."""
    return "detector" if N_obs * N_Tu - 4 * N_p >= 0 else "beam"


def gather_pixels(local, dist, group=None):
    """Concatenate per-rank pixel blocks (leading dimension) on every rank."""
    import torch
    world = dist.get_world_size(group)
    sizes = [None] * world
    dist.all_gather_object(sizes, int(local.shape[0]), group=group)
    mx = max(sizes)
    pad = torch.zeros((mx,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    return torch.cat([b[:s] for b, s in zip(bufs, sizes)], dim=0)


def reduce_beam(local, dist, group=None):
    """Sum per-rank records in place (beam parallelization)."""
    dist.all_reduce(local, op=dist.ReduceOp.SUM, group=group)
    return local
