"""Pixel-sharded transforms across ranks (the multi-GPU design), on CPU.

Two gloo ranks each own a band of SLM rows (paper_2505_08777_gb300.shard).
Each computes the oracle's forward partial sums over its rows; one
all-reduce of the N spot fields must equal the unsharded forward, the
adjoint is local per pixel, and a whole sharded WGS run (forward
all-reduce, replicated spot update, local adjoint) must reproduce the
unsharded oracle's phase and weights."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2505_08777_gb300.shard import row_block, row_blocks  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from workloads import random_problem
    return random_problem(17, 48, 80, 23, list(range(2, 12)), defocus_max=6.0)


def _allreduce_complex(x: np.ndarray) -> np.ndarray:
    t = torch.from_numpy(np.stack([x.real, x.imag]))
    dist.all_reduce(t)
    return t[0].numpy() + 1j * t[1].numpy()


def _worker(rank: int, world: int, port: int, out_dir: str):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import transform, wgs, zernike
        p = _problem()
        Z = zernike.basis(p.nx, p.ny, p.noll)
        C = p.coeff.astype(np.float64)
        A = p.amp.astype(np.float64).ravel()
        r0, r1 = row_block(p.ny, rank, world)
        own = np.arange(r0 * p.nx, r1 * p.nx)          # this rank's pixels (row-major)
        # forward: partial sums over own rows, then one all-reduce
        f = transform.field(A, p.phase0.ravel().astype(np.float64))
        E = _allreduce_complex(transform.forward(f[own], C, Z[:, own]))
        # adjoint: local per pixel
        rng = np.random.default_rng(3)
        y = rng.normal(size=p.N) + 1j * rng.normal(size=p.N)
        g_own = transform.adjoint(y, C, Z[:, own])
        # sharded WGS: forward all-reduce, replicated update, local adjoint
        phase = p.phase0.ravel().astype(np.float64)[own].copy()
        w = p.target.astype(np.float64).copy()
        for _ in range(6):
            Ew = _allreduce_complex(transform.forward(transform.field(A[own], phase), C, Z[:, own]))
            w, yw = wgs.weight_update(Ew, w, p.target)
            phase = transform.phase_of(transform.adjoint(yw, C, Z[:, own]))
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), E=E, g_own=g_own, own=own, phase=phase, w=w, y=y)
    finally:
        dist.destroy_process_group()


def test_row_blocks_cover_in_whole_tile_bands():
    for ny in (1, 31, 32, 33, 80, 1152):
        for world in (1, 2, 3, 8):
            blocks = row_blocks(ny, world)
            assert blocks[0][0] == 0 and blocks[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            assert all(r0 % 32 == 0 and (r1 % 32 == 0 or r1 == ny) for r0, r1 in blocks)
    assert row_blocks(80, 2) == [(0, 32), (32, 80)]
    with pytest.raises(ValueError):
        row_blocks(10, 0)


def test_two_rank_sharded_transforms_equal_unsharded(tmp_path):
    from oracle import transform, wgs, zernike
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    p = _problem()
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    A = p.amp.astype(np.float64).ravel()
    E_ref = transform.forward(transform.field(A, p.phase0.ravel().astype(np.float64)), C, Z)
    for r in res:   # every rank holds the full spot fields after the all-reduce
        np.testing.assert_allclose(r["E"], E_ref, rtol=1e-12, atol=1e-12 * np.abs(E_ref).max())
    g_ref = transform.adjoint(res[0]["y"], C, Z)
    g = np.zeros_like(g_ref)
    for r in res:
        g[r["own"]] = r["g_own"]
    np.testing.assert_allclose(g, g_ref, rtol=1e-12, atol=1e-12 * np.abs(g_ref).max())
    ref = wgs.run(A, p.phase0, C, Z, p.target, 6)
    phase = np.zeros(p.M)
    for r in res:
        phase[r["own"]] = r["phase"]
        np.testing.assert_allclose(r["w"], ref.weights, rtol=1e-9)
    np.testing.assert_allclose(np.exp(1j * phase), np.exp(1j * ref.phase), atol=1e-8)
