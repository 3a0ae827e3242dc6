"""GPU parity of the forward / adjoint transforms against the oracle.

Every case calls the CUDA library through the C ABI (Hologram binding) and
compares with the complex128 oracle on the same seeded inputs, normwise and
with a per-element guard, at tolerance 1e-4 (the bound for spot and SLM
fields of one pass).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import GRAD_TOL, REL_TOL, assert_close, basis_at, oracle_forward, oracle_inputs  # noqa: E402
from oracle import grad as ograd, transform, zernike  # noqa: E402
from workloads import config_c1, config_c2, config_c3, random_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _holo(p, basis=None):
    from paper_2505_08777_gb300 import Hologram
    amp = torch.from_numpy(p.amp).cuda()
    coeff = torch.from_numpy(p.coeff).cuda()
    if basis is not None:
        return Hologram(amp, coeff, basis=torch.from_numpy(basis.astype(np.float32)).cuda())
    return Hologram(amp, coeff, noll=p.noll)


def _rand_complex(rng, shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)


def test_forward_c1():
    p = config_c1(1)
    h = _holo(p)
    E = h.forward(torch.from_numpy(p.phase0).cuda()).cpu().numpy()
    ref = oracle_forward(p, p.phase0)
    assert_close(E, ref, what="forward c1")


CASES = [
    # (nx, ny, N, noll, defocus_max) : ragged tiles, chunk and batch tails, every D range
    (97, 61, 37, list(range(2, 12)), 5.0),
    (33, 32, 300, list(range(2, 13)), 20.0),
    (64, 40, 17, [2, 3, 4, 5, 6], 10.0),
    (45, 77, 5, [2, 3], 0.0),
    (50, 50, 260, [4], 20.0),
    (70, 31, 33, list(range(2, 18)), 3.0),
    (1, 1, 1, [2, 3, 4], 1.0),
    (40, 130, 9, [2, 3, 4, 5, 6, 7, 8], 2.0),
    (9, 20, 70, [2, 3, 4, 5, 6, 7, 8, 9, 10], 2.0),
]


@pytest.mark.parametrize("nx,ny,N,noll,dmax", CASES)
def test_forward_adjoint_ragged(nx, ny, N, noll, dmax):
    p = random_problem(100 + nx + ny + N, nx, ny, N, noll, defocus_max=dmax)
    h = _holo(p)
    Z, C, A = oracle_inputs(p)
    E = h.forward(torch.from_numpy(p.phase0).cuda()).cpu().numpy()
    assert_close(E, transform.forward(transform.field(A, p.phase0), C, Z), what="forward")
    rng = np.random.default_rng(nx * 7 + N)
    y = _rand_complex(rng, N)
    g, ph = h.adjoint(torch.from_numpy(y).cuda(), want_field=True, want_phase=True)
    g_ref = transform.adjoint(y.astype(np.complex128), C, Z)
    assert_close(g.cpu().numpy(), g_ref, what="adjoint")
    # phase projection compared through unit phasors weighted by |g|
    u = np.exp(1j * ph.cpu().numpy().astype(np.float64).ravel())
    u_ref = np.exp(1j * transform.phase_of(g_ref))
    w = np.abs(g_ref)
    assert np.linalg.norm(w * (u - u_ref)) <= REL_TOL * np.linalg.norm(w)


def test_forward_field_and_adjoint_identity():
    p = random_problem(7, 80, 72, 50, list(range(2, 12)), defocus_max=10.0)
    h = _holo(p)
    Z, C, _ = oracle_inputs(p)
    rng = np.random.default_rng(3)
    x = _rand_complex(rng, (p.ny, p.nx))
    y = _rand_complex(rng, p.N)
    Kx = h.forward_field(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
    Khy, _ = h.adjoint(torch.from_numpy(y).cuda())
    Khy = Khy.cpu().numpy().astype(np.complex128).ravel()
    assert_close(Kx, transform.forward(x.ravel().astype(np.complex128), C, Z), what="forward_field")
    lhs = np.vdot(y.astype(np.complex128), Kx)
    rhs = np.vdot(Khy, x.ravel().astype(np.complex128))
    scale = np.linalg.norm(Kx) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_user_basis_matches_zernike_path():
    p = random_problem(9, 96, 64, 40, list(range(2, 12)), defocus_max=5.0)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    h_n = _holo(p)
    h_b = _holo(p, basis=Z.reshape(len(p.noll), p.ny, p.nx))
    ph = torch.from_numpy(p.phase0).cuda()
    E_n = h_n.forward(ph).cpu().numpy()
    E_b = h_b.forward(ph).cpu().numpy()
    ref = transform.forward(transform.field(p.amp.astype(np.float64), p.phase0),
                            p.coeff.astype(np.float64), Z.astype(np.float32).astype(np.float64))
    assert_close(E_b, ref, what="user basis")
    assert_close(E_n, E_b, what="noll vs user basis")


@pytest.mark.parametrize("variant", [0, 2])
def test_user_basis_adjoint_and_gradients(variant):
    # a caller basis has no polynomial form, so dL/dC runs on the FMA moment
    # kernel; the adjoint and dL/dphi on the family the variant picks
    p = random_problem(19, 112, 80, 300, list(range(2, 12)), defocus_max=4.0)
    Z32 = zernike.basis(p.nx, p.ny, p.noll).astype(np.float32)
    h = _holo(p, basis=Z32.reshape(len(p.noll), p.ny, p.nx))
    h.set_variant(variant)
    Z, C = Z32.astype(np.float64), p.coeff.astype(np.float64)
    A = p.amp.astype(np.float64).ravel()
    rng = np.random.default_rng(4)
    y = _rand_complex(rng, p.N)
    g, _ = h.adjoint(torch.from_numpy(y).cuda())
    assert_close(g.cpu().numpy(), transform.adjoint(y.astype(np.complex128), C, Z), what="user basis adjoint")
    E = transform.forward(transform.field(A, p.phase0), C, Z)
    gE = ograd.grad_E(E, p.target).astype(np.complex64)
    dph, dC = h.grad(torch.from_numpy(p.phase0).cuda(), torch.from_numpy(gE).cuda())
    dph_ref, dC_ref = ograd.backward(A, p.phase0, C, Z, gE.astype(np.complex128))
    assert np.linalg.norm(dph.cpu().numpy().ravel() - dph_ref) <= GRAD_TOL * np.linalg.norm(dph_ref)
    assert np.linalg.norm(dC.cpu().numpy() - dC_ref) <= GRAD_TOL * np.linalg.norm(dC_ref)
    assert not (h.launch_info()["kernels"] & 8)   # no tensor-core moments for a caller basis


def test_coefficients_round_trip():
    p = random_problem(24, 64, 48, 30, [2, 3, 4, 5, 6])
    h = _holo(p)
    np.testing.assert_array_equal(h.coefficients().cpu().numpy(), p.coeff)
    C2 = torch.from_numpy(p.coeff * 0.5).cuda()
    h.set_coefficients(C2)
    got = h.coefficients()
    assert torch.equal(got, C2) and got.data_ptr() != C2.data_ptr()


def test_set_amplitude_changes_the_nearfield():
    p = random_problem(23, 96, 72, 60, list(range(2, 12)))
    h = _holo(p)
    ph = torch.from_numpy(p.phase0).cuda()
    rng = np.random.default_rng(8)
    amp2 = rng.uniform(0.2, 1.0, size=p.amp.shape).astype(np.float32)
    h.set_amplitude(torch.from_numpy(amp2).cuda())
    Z, C, _ = oracle_inputs(p)
    ref = transform.forward(transform.field(amp2.astype(np.float64).ravel(), p.phase0), C, Z)
    assert_close(h.forward(ph).cpu().numpy(), ref, what="forward after set_amplitude")
    h.set_amplitude(torch.from_numpy(p.amp).cuda())
    assert_close(h.forward(ph).cpu().numpy(), oracle_forward(p, p.phase0), what="amplitude restored")


def test_phase_conjugate_focus_and_flat_phase():
    # closed forms on the GPU path: C = 0, phase 0 -> E = sum A; conjugate hologram focuses spot n
    p = random_problem(5, 128, 96, 8, list(range(2, 12)), defocus_max=10.0)
    Z, C, A = oracle_inputs(p)
    h = _holo(p)
    n = 3
    phase = (C[n] @ Z).reshape(p.ny, p.nx).astype(np.float32)
    E = h.forward(torch.from_numpy(phase).cuda()).cpu().numpy()
    assert abs(E[n] - A.sum()) <= 1e-4 * A.sum()
    p0 = random_problem(5, 128, 96, 4, list(range(2, 12)))
    p0.coeff[:] = 0
    h0 = _holo(p0)
    E0 = h0.forward(torch.zeros(p0.ny, p0.nx, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(E0, np.full(4, p0.amp.astype(np.float64).sum()), rtol=1e-5)


def test_integer_bin_tilt_equals_fft_bin_on_gpu():
    nx, ny = 128, 64
    R = min(nx, ny) / 2.0
    bins = [(0, 0), (5, -3), (-17, 9), (40, 20), (-63, -31)]
    C = np.array([[2 * math.pi * kx * R / nx, 2 * math.pi * ky * R / ny] for kx, ky in bins], np.float32)
    rng = np.random.default_rng(0)
    f = _rand_complex(rng, (ny, nx))
    from paper_2505_08777_gb300 import Hologram
    h = Hologram(torch.ones(ny, nx, device="cuda"), torch.from_numpy(C).cuda(), noll=[2, 3])
    E = h.forward_field(torch.from_numpy(f).cuda()).cpu().numpy()
    F = np.fft.fft2(f.astype(np.complex128))
    ref = np.array([F[ky % ny, kx % nx] * np.exp(1j * math.pi * (kx * (nx - 1) / nx + ky * (ny - 1) / ny))
                    for kx, ky in bins])
    # the FP32 coefficient differs from the exact bin by its rounding; compare with the oracle's
    # value at the same FP32 coefficients and with the FFT bin at a looser bound
    Z = zernike.basis(nx, ny, [2, 3])
    assert_close(E, transform.forward(f.ravel().astype(np.complex128), C.astype(np.float64), Z), what="fft case")
    assert np.linalg.norm(E - ref) <= 1e-3 * np.linalg.norm(ref)


def test_determinism():
    p = random_problem(11, 200, 150, 120, list(range(2, 12)), defocus_max=5.0)
    h = _holo(p)
    ph = torch.from_numpy(p.phase0).cuda()
    E1 = h.forward(ph).cpu().numpy()
    E2 = h.forward(ph).cpu().numpy()
    assert np.array_equal(E1.view(np.uint32), E2.view(np.uint32))


@pytest.mark.parametrize("make", [config_c2, config_c3], ids=["c2_1024x1024_N400", "c3_1920x1152_N2000"])
def test_full_size_sampled(make):
    """At the benchmark sizes: forward on sampled spots and adjoint on sampled
    pixels, each checked against the oracle computed for those entries only."""
    p = make(1)
    h = _holo(p)
    rng = np.random.default_rng(42)
    ph = torch.from_numpy(p.phase0).cuda()
    E = h.forward(ph).cpu().numpy()
    idx = np.sort(rng.choice(p.N, size=12, replace=False))
    Z = zernike.basis(p.nx, p.ny, p.noll)
    ref = oracle_forward(p, p.phase0, Z=Z, idx=idx, workers=8)
    assert_close(E[idx], ref, what="forward sampled")
    y = _rand_complex(rng, p.N)
    g, _ = h.adjoint(torch.from_numpy(y).cuda())
    g = g.cpu().numpy().ravel()
    pix = np.sort(rng.choice(p.M, size=4096, replace=False))
    g_ref = transform.adjoint(y.astype(np.complex128), p.coeff.astype(np.float64), basis_at(p, pix))
    assert_close(g[pix], g_ref, what="adjoint sampled")


@pytest.mark.parametrize("nx,ny,N,noll,dmax", [(97, 61, 37, list(range(2, 12)), 5.0), (160, 128, 300, list(range(2, 13)), 20.0),
                                                (128, 96, 150, [4, 5, 2, 6, 7, 3, 8, 9, 10, 11, 12], 10.0),
                                                (96, 96, 70, list(range(4, 15)), 6.0),
                                                (64, 40, 17, [2, 3, 4, 5, 6], 10.0), (33, 70, 5, [4], 20.0),
                                                (256, 256, 400, list(range(2, 12)), 8.0)])
def test_adjoint_kernel_variants_agree_with_oracle(nx, ny, N, noll, dmax):
    """FMA-pipe adjoint (variant 1) and tensor-core adjoint (variant 2, split-tf32
    phase contraction) against the oracle, on the same inputs."""
    p = random_problem(200 + nx + N, nx, ny, N, noll, defocus_max=dmax)
    h = _holo(p)
    Z, C, _ = oracle_inputs(p)
    rng = np.random.default_rng(N)
    y = _rand_complex(rng, N)
    g_ref = transform.adjoint(y.astype(np.complex128), C, Z)
    errs = {}
    for variant in (1, 2):
        h.set_variant(variant)
        g, ph = h.adjoint(torch.from_numpy(y).cuda(), want_field=True, want_phase=True)
        errs[variant] = assert_close(g.cpu().numpy(), g_ref, what=f"adjoint variant {variant}")
    print("adjoint normwise/max-guard errors by variant:", errs)


@pytest.mark.parametrize("nx,ny,N,noll,dmax", [(97, 61, 37, list(range(2, 12)), 5.0), (160, 128, 300, list(range(2, 13)), 20.0),
                                                (128, 96, 150, [4, 5, 2, 6, 7, 3, 8, 9, 10, 11, 12], 10.0),
                                                (96, 96, 70, list(range(4, 15)), 6.0),
                                                (64, 40, 17, [2, 3, 4, 5, 6], 10.0), (33, 70, 5, [4], 20.0),
                                                (256, 256, 400, list(range(2, 12)), 8.0)])
def test_forward_kernel_variants_agree_with_oracle(nx, ny, N, noll, dmax):
    """FMA-pipe forward (variant 1) and tensor-core forward (variant 2) against
    the oracle, for phase-only and general complex nearfields."""
    p = random_problem(300 + nx + N, nx, ny, N, noll, defocus_max=dmax)
    h = _holo(p)
    Z, C, A = oracle_inputs(p)
    rng = np.random.default_rng(N + 1)
    x = _rand_complex(rng, (p.ny, p.nx))
    E_ref = transform.forward(transform.field(A, p.phase0), C, Z)
    Ef_ref = transform.forward(x.ravel().astype(np.complex128), C, Z)
    for variant in (1, 2):
        h.set_variant(variant)
        E = h.forward(torch.from_numpy(p.phase0).cuda()).cpu().numpy()
        assert_close(E, E_ref, what=f"forward variant {variant}")
        Ef = h.forward_field(torch.from_numpy(x).cuda()).cpu().numpy()
        assert_close(Ef, Ef_ref, what=f"forward_field variant {variant}")


@pytest.mark.parametrize("N", [530, 560])
def test_forward_with_ranges_claimed_by_sm(N):
    """A replicated last spot block (N mod 128 <= 64) on a grid large enough
    that the tensor-core forward claims its CTA ranges by SM (every range of
    32 chunks or more): against the oracle, bitwise identical over repeated
    launches (which CTA runs a range changes, each range's arithmetic does
    not), forward after forward, and with no error raised."""
    p = random_problem(900 + N, 512, 512, N, list(range(2, 12)), defocus_max=6.0)
    h = _holo(p)
    li = h.launch_info()
    assert li["kernels"] & 4 and li["split_flags"] & 8   # tensor-core forward, ranges claimed by SM
    ph = torch.from_numpy(p.phase0).cuda()
    outs = [h.forward(ph).cpu().numpy() for _ in range(4)]
    torch.cuda.synchronize()
    h.check()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert_close(outs[0], oracle_forward(p, p.phase0, workers=8), what=f"forward N={N} (ranges claimed by SM)")
