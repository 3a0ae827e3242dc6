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


def band_holograms(amp, coeff, noll, ny_full: int, blocks, stream=None):
    """Band handles of one hologram for the row ranges `blocks` ([r0, r1)
    pairs from row_blocks; empty ranges are skipped): amp is this process's
    full-width rows of the amplitude, (ny_full, nx) when several bands of the
    same process cut it, each band taking its own rows."""
    from .hologram import Hologram
    out = []
    for r0, r1 in blocks:
        if r1 > r0:
            out.append(Hologram(amp[r0:r1].contiguous(), coeff, noll=noll, row0=r0, ny_full=ny_full,
                                stream=stream))
    return out


def sharded_wgs(bands, phases, weights, target, iters: int, allreduce=None, sum_a2: float = 0.0, stream=None):
    """Weighted GS over pixel bands (Sec. II / Sec. III, sharded by Methods'
    per-pixel independence): every iteration, the forward partial spot fields
    of each band, summed over the bands and the ranks (one all-reduce of N
    complex64), the spot update (replicated: every rank computes the same w
    and y from the same E), then each band's local adjoint writing its phase.
    One more forward gives the returned E and metrics.

    bands: this process's band handles (one per GPU rank in a multi-GPU run;
    several on one device stand for several ranks); phases: their (rows, nx)
    phases, updated in place; weights: (N,) updated in place; allreduce(E):
    sums E over the ranks in place (e.g. torch.distributed.all_reduce under
    NCCL), None with a single process; sum_a2: sum of A^2 over the whole
    grid for the efficiency (0: the first band's own)."""
    import torch
    N = bands[0].N
    dev = phases[0].device
    E = torch.empty(N, dtype=torch.complex64, device=dev)
    part = torch.empty_like(E) if len(bands) > 1 else None
    y = torch.empty_like(E)

    def forward_all():
        bands[0].forward(phases[0], out=E, stream=stream)
        for b, ph in zip(bands[1:], phases[1:]):
            # several bands in one process: their sum stands in for the
            # all-reduce between ranks
            b.forward(ph, out=part, stream=stream)
            E.add_(part)
        if allreduce is not None:
            allreduce(E)

    forward_all()
    for _ in range(iters):
        bands[0].spot_update(E, weights, target, out=y, stream=stream)
        for b, ph in zip(bands, phases):
            b.adjoint(y, want_field=False, phase_out=ph, stream=stream)
        forward_all()
    met = bands[0].spot_metrics(E, target, sum_a2, stream=stream)
    return E, met
