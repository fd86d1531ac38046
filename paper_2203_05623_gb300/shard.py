"""Distribution of perturbations over ranks (one process per GPU).

Every (state, perturbation) Sternheimer system is independent (Sec. 3), so a batch
of perturbations is split over ranks with no exchange on the data path; the paper
distributes perturbations over its "images" block-cyclically (Sec. 4).  Rank r owns
the blocks r, r + world, r + 2 world, ... of `block` consecutive perturbations.
"""
from __future__ import annotations


def owned_perturbations(n_global: int, rank: int, world: int, block: int = 1) -> list[int]:
    """Indices of the perturbations owned by `rank` (block-cyclic, in increasing order)."""
    if world < 1 or not (0 <= rank < world) or block < 1 or n_global < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, block >= 1, n_global >= 0")
    out = []
    for b0 in range(rank * block, n_global, world * block):
        out.extend(range(b0, min(b0 + block, n_global)))
    return out
