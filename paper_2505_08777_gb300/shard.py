"""Pixel sharding of one hologram over several ranks (host logic only).

The transforms are sums over pixels (forward) or independent per pixel
(adjoint), so a hologram shards by contiguous blocks of SLM rows: each rank
computes the forward's partial spot fields over its rows, one all-reduce of
the N complex spot fields (at most a few tens of KB) completes E, the spot
update is replicated on every rank, and the adjoint needs no communication
(paper, Methods "Computational Scaling": every pixel's kernel values depend
only on that pixel and the global N x D coefficient matrix). Blocks are cut
at whole 32-row tile rows so that each rank's tiles, and their anchor
pixels, are tiles of the full grid.
"""
from __future__ import annotations

TILE_ROWS = 32


def row_blocks(ny: int, world: int, align: int = TILE_ROWS) -> list[tuple[int, int]]:
    """[r0, r1) row ranges of `world` ranks: whole `align`-row bands, as even
    as possible, covering [0, ny) in order (a rank may get an empty range
    when there are fewer bands than ranks)."""
    if ny < 0 or world < 1 or align < 1:
        raise ValueError("need ny >= 0, world >= 1, align >= 1")
    bands = (ny + align - 1) // align
    out = []
    for r in range(world):
        b0, b1 = bands * r // world, bands * (r + 1) // world
        out.append((min(ny, b0 * align), min(ny, b1 * align)))
    return out


def row_block(ny: int, rank: int, world: int, align: int = TILE_ROWS) -> tuple[int, int]:
    """This rank's [r0, r1) row range (see row_blocks)."""
    return row_blocks(ny, world, align)[rank]
