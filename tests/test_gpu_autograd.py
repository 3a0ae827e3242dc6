"""torch.autograd.Function over the hand-written gradient kernels.

Gradients of the spot-intensity loss through spot_field are compared with
(a) the oracle's closed form (pinned to float64 finite differences in the
CPU tests) and (b) plain PyTorch float64 on the GPU applied to the explicit
kernel matrix of the same small problem, at 1e-3 normwise; a few Adam steps
must lower the loss.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import GRAD_TOL, oracle_inputs  # noqa: E402
from oracle import grad as ograd  # noqa: E402
from workloads import random_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _setup(seed=4, nx=80, ny=72, N=48, noll=tuple(range(2, 12))):
    from paper_2505_08777_gb300 import Hologram
    p = random_problem(seed, nx, ny, N, list(noll), defocus_max=5.0, target_range=(0.5, 1.5))
    h = Hologram(torch.from_numpy(p.amp).cuda(), torch.from_numpy(p.coeff).cuda(), noll=p.noll)
    return p, h


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_autograd_matches_oracle_and_torch_reference():
    from paper_2505_08777_gb300.autograd import spot_field, spot_intensity_loss
    p, h = _setup()
    phase = torch.from_numpy(p.phase0).cuda().requires_grad_(True)
    coeff = torch.from_numpy(p.coeff).cuda().requires_grad_(True)
    t = torch.from_numpy(p.target).cuda()
    loss = spot_intensity_loss(spot_field(h, phase, coeff), t)
    loss.backward()
    Z, C, A = oracle_inputs(p)
    L_ref, dphi_ref, dC_ref = ograd.grad(A, p.phase0.astype(np.float64).ravel(), C, Z, p.target)
    assert abs(loss.item() - L_ref) <= 1e-3 * abs(L_ref)
    assert _rel(phase.grad.cpu().numpy().astype(np.float64).ravel(), dphi_ref) <= GRAD_TOL
    assert _rel(coeff.grad.cpu().numpy().astype(np.float64), dC_ref) <= GRAD_TOL
    # plain PyTorch float64 reference of the same operation (explicit kernel matrix)
    ph64 = torch.from_numpy(p.phase0.astype(np.float64)).cuda().requires_grad_(True)
    C64 = torch.from_numpy(C).cuda().requires_grad_(True)
    Z64 = torch.from_numpy(Z).cuda()
    A64 = torch.from_numpy(A).cuda()
    E64 = torch.exp(-1j * (C64 @ Z64)) @ (A64 * torch.exp(1j * ph64.reshape(-1)))
    I = E64.abs() ** 2
    r = I / I.mean() - torch.from_numpy(p.target.astype(np.float64)).cuda()
    (r * r).sum().backward()
    assert _rel(phase.grad.double().cpu().numpy().ravel(), ph64.grad.cpu().numpy().ravel()) <= GRAD_TOL
    assert _rel(coeff.grad.double().cpu().numpy(), C64.grad.cpu().numpy()) <= GRAD_TOL


def test_one_handle_two_coefficient_sets_in_one_graph():
    # two forwards on one handle with different C, then one backward: the
    # second backward to run finds the handle holding the other C and must
    # set its own again (the handle counts set_coefficients calls)
    from paper_2505_08777_gb300.autograd import spot_field, spot_intensity_loss
    p, h = _setup(seed=6)
    rng = np.random.default_rng(3)
    C2np = (p.coeff + rng.normal(0.0, 0.3, p.coeff.shape)).astype(np.float32)
    phase = torch.from_numpy(p.phase0).cuda().requires_grad_(True)
    c1 = torch.from_numpy(p.coeff).cuda().requires_grad_(True)
    c2 = torch.from_numpy(C2np).cuda().requires_grad_(True)
    t = torch.from_numpy(p.target).cuda()
    loss = spot_intensity_loss(spot_field(h, phase, c1), t) + spot_intensity_loss(spot_field(h, phase, c2), t)
    loss.backward()
    Z, C1, A = oracle_inputs(p)
    ph = p.phase0.astype(np.float64).ravel()
    L1, dphi1, dC1 = ograd.grad(A, ph, C1, Z, p.target)
    L2, dphi2, dC2 = ograd.grad(A, ph, C2np.astype(np.float64), Z, p.target)
    assert abs(loss.item() - (L1 + L2)) <= 1e-3 * abs(L1 + L2)
    assert _rel(c1.grad.cpu().numpy().astype(np.float64), dC1) <= GRAD_TOL
    assert _rel(c2.grad.cpu().numpy().astype(np.float64), dC2) <= GRAD_TOL
    assert _rel(phase.grad.cpu().numpy().astype(np.float64).ravel(), dphi1 + dphi2) <= GRAD_TOL


def test_adam_lowers_spot_loss():
    from paper_2505_08777_gb300.autograd import spot_field, spot_intensity_loss
    p, h = _setup(seed=9, nx=96, ny=96, N=64)
    phase = torch.from_numpy(p.phase0).cuda().requires_grad_(True)
    coeff = torch.from_numpy(p.coeff).cuda().requires_grad_(True)
    t = torch.from_numpy(p.target).cuda()
    opt = torch.optim.Adam([phase, coeff], lr=0.05)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        loss = spot_intensity_loss(spot_field(h, phase, coeff), t)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < 0.25 * losses[0], losses[::5]


def test_gradient_only_for_requested_inputs():
    from paper_2505_08777_gb300.autograd import spot_field
    p, h = _setup(seed=2, N=10)
    phase = torch.from_numpy(p.phase0).cuda().requires_grad_(True)
    E = spot_field(h, phase)        # coefficients fixed
    (E.abs() ** 2).sum().backward()
    assert phase.grad is not None and torch.isfinite(phase.grad).all()


def test_step_is_graph_capturable_and_bitwise_eager():
    # every library call is stream-ordered and allocation-free, so a whole
    # forward + backward captures as one CUDA graph; the kernels are
    # deterministic, so a replay gives the eager gradients bit for bit
    from paper_2505_08777_gb300.autograd import spot_field, spot_intensity_loss
    p, h = _setup(seed=9, nx=96, ny=80, N=150)
    ph = torch.from_numpy(p.phase0).cuda().requires_grad_(True)
    C = torch.from_numpy(p.coeff).cuda().requires_grad_(True)
    t = torch.from_numpy(p.target).cuda()

    def step():
        ph.grad = None if ph.grad is None else ph.grad.zero_()
        C.grad = None if C.grad is None else C.grad.zero_()
        loss = spot_intensity_loss(spot_field(h, ph, C), t)
        loss.backward()
        return loss.detach()

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            step()
    torch.cuda.current_stream().wait_stream(side)
    L_eager = step().clone()
    g_ph, g_C = ph.grad.clone(), C.grad.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        L_static = step()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(L_static, L_eager)
    assert torch.equal(ph.grad, g_ph) and torch.equal(C.grad, g_C)


def test_spot_loss_kernel_matches_float64_autograd():
    # the library's loss and dL/dE against float64 torch autograd of the
    # written-out loss, on random fields (sizes past one CTA's 1024 threads)
    from paper_2505_08777_gb300.hologram import spot_loss
    rng = np.random.default_rng(12)
    for N in (7, 1024, 5000):
        E = (rng.normal(size=N) + 1j * rng.normal(size=N)).astype(np.complex64)
        t = rng.uniform(0.5, 1.5, size=N).astype(np.float32)
        L, g = spot_loss(torch.from_numpy(E).cuda(), torch.from_numpy(t).cuda())
        E64 = torch.from_numpy(E.astype(np.complex128)).requires_grad_(True)
        I = E64.abs() ** 2
        r = I / I.mean() - torch.from_numpy(t.astype(np.float64))
        L64 = (r * r).sum()
        L64.backward()
        assert abs(L.item() - L64.item()) <= 1e-5 * abs(L64.item())
        assert _rel(g.cpu().numpy().astype(np.complex128), E64.grad.numpy()) <= 1e-5
        # and the oracle's closed form of the same gradient
        assert _rel(g.cpu().numpy().astype(np.complex128), ograd.grad_E(E.astype(np.complex128), t)) <= 1e-5
