"""Host-side logic of running independent replicas on N devices.

Monte Carlo trajectories are independent (Secs. I, V), so N devices run
disjoint trajectory ranges of the same seed and nothing crosses devices on
the data path.  What crosses them is the end of a job: each rank's
sufficient statistics are gathered to rank 0 and merged exactly
(mctrg_merge_estimates), and the slowest rank's time is the job's time.
"""
from . import mctrg

# Estimate fields that the merge reads (the rest follows from them).
_FIELDS = ("n", "ln_scale", "sum_x", "m2_x", "n_negative", "n_flagged")


def first_trajectory(step, rank, world, per_step):
    """First trajectory counter of (step, rank): rank r at step s runs
    [(s * world + r) * per_step, ... + per_step), so every counter is used
    once whatever the number of ranks."""
    return (step * world + rank) * per_step


def pack(estimates):
    """Sufficient statistics of a list of estimates as a flat list of floats."""
    out = []
    for e in estimates:
        out.extend(float(getattr(e, f)) for f in _FIELDS)
    return out


def unpack(values):
    """Inverse of pack: mctrg.Estimate structures (only the merge fields set)."""
    k = len(_FIELDS)
    ests = []
    for i in range(0, len(values), k):
        e = mctrg.Estimate()
        for f, v in zip(_FIELDS, values[i:i + k]):
            setattr(e, f, int(round(v)) if f in ("n", "n_negative", "n_flagged") else float(v))
        ests.append(e)
    return ests


def gather_estimates(dist, estimates, device="cpu"):
    """Every rank's estimates, gathered to all ranks in rank order (each rank
    passes the same number).  dist is torch.distributed with an initialized
    process group (gloo on host tensors, NCCL on device tensors)."""
    import torch
    local = torch.tensor(pack(estimates), dtype=torch.float64, device=device)
    parts = [torch.empty_like(local) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, local)
    out = []
    for p in parts:
        out.extend(unpack(p.cpu().tolist()))
    return out
