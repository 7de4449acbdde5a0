"""Differentiation through hierarchization: the adjoint kernel (transpose of
Alg. 1) behind torch.autograd.  Checked by the dot-product test
<Hx, y> = <x, H^T y> and by central finite differences of the weighted
surplus loss L = sum_i w_i alpha_i^2, w = 2^{-|level(i)|_1}, on the
differentiation workload (16 grids of level (8,8,8))."""
import numpy as np
import pytest

import oracle
from paper_1309_0392_gb300 import inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")
from paper_1309_0392_gb300.autograd import DehierarchizeFn, HierarchizeFn  # noqa: E402

pytestmark = pytest.mark.gpu


def level_weights_torch(levels, device):
    """w = prod_k 2^{-level_k(i_k)} as a flat tensor (dimension 0 fastest)."""
    w = torch.ones(1, dtype=torch.float64, device=device)
    for l in reversed(levels):
        lev = np.zeros(2 ** l + 1)
        for i in range(1, 2 ** l):
            lev[i] = l - ((i & -i).bit_length() - 1)
        w = torch.kron(w, torch.tensor(2.0 ** -lev, device=device))
    return w


def test_level_weights_match_oracle():
    for levels in [(3, 2), (2, 3, 1), (5,)]:
        assert np.array_equal(level_weights_torch(levels, "cuda").cpu().numpy(), oracle.level_weights(levels))


@pytest.mark.parametrize("levels,batch", [((6, 5, 4), None), ((5, 4, 4, 3), None), ((4, 4, 4), 3), ((7, 7), None)])
def test_adjoint_matches_oracle(levels, batch):
    B = batch or 1
    n = inputs.num_points(levels)
    y = np.random.default_rng(2).uniform(-1, 1, (B, n))
    t = torch.tensor(y.reshape(-1), device="cuda")
    gbh.hierarchize_adjoint(t, levels, batch=batch)
    got = t.cpu().numpy().reshape(B, n)
    for b in range(B):
        ref = oracle.hierarchize_adjoint(y[b], levels)
        assert np.abs(got[b] - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1.0)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_dot_product_full_workload(dtype, tol):
    levels, u = inputs.cfg5()
    B = u.shape[0]
    x = torch.tensor(u.reshape(-1), dtype=dtype, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(11)
    y = (torch.rand(x.numel(), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1).to(dtype)
    hx = x.clone()
    gbh.hierarchize(hx, levels, batch=B)
    hty = y.clone()
    gbh.hierarchize_adjoint(hty, levels, batch=B)
    lhs = torch.dot(hx.double(), y.double()).item()
    rhs = torch.dot(x.double(), hty.double()).item()
    assert abs(lhs - rhs) <= tol * hx.double().norm().item() * y.double().norm().item()


def test_autograd_gradient_matches_oracle():
    levels, B = (4, 3, 3), 2
    u = np.random.default_rng(3).uniform(-1, 1, (B, inputs.num_points(levels)))
    w = oracle.level_weights(levels)
    t = torch.tensor(u, device="cuda", requires_grad=True)
    alpha = HierarchizeFn.apply(t, levels)
    loss = (torch.tensor(w, device="cuda") * alpha ** 2).sum()
    loss.backward()
    for b in range(B):
        ref = oracle.hierarchize_adjoint(2.0 * w * oracle.hierarchize(u[b], levels), levels)
        assert np.abs(t.grad[b].cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    # the input is untouched by the forward
    assert np.array_equal(t.detach().cpu().numpy(), u)


def test_central_differences_full_workload():
    """FD on 64 coordinates (half at coarse, half at fine levels).  The loss is
    quadratic in u, so central differences have no truncation error for any
    step; a unit step keeps the rounding of the loss far below the signal.
    Only the perturbed grid's loss term changes, so only it is re-evaluated."""
    levels, u = inputs.cfg5()
    B, n = u.shape
    w = level_weights_torch(levels, "cuda")
    x = torch.tensor(u, device="cuda", requires_grad=True)
    alpha = HierarchizeFn.apply(x, levels)
    loss = (w * alpha ** 2).sum()
    loss.backward()
    g = x.grad.detach()
    gmax = g.abs().max().item()

    lev_sum = torch.log2(w).neg()                      # |level(i)|_1 per point
    rng = np.random.default_rng(64)
    coarse = torch.nonzero(lev_sum <= 6).flatten().cpu().numpy()
    fine = torch.nonzero(lev_sum >= 18).flatten().cpu().numpy()
    picks = [(int(rng.integers(B)), int(c)) for c in rng.choice(coarse, 32, replace=False)]
    picks += [(int(rng.integers(B)), int(f)) for f in rng.choice(fine, 32, replace=False)]

    def grid_loss(vec):
        a = vec.clone()
        gbh.hierarchize(a, levels)
        return (w * a * a).sum().item()

    eps = 1.0
    for b, c in picks:
        base = x.detach()[b]
        up, dn = base.clone(), base.clone()
        up[c] += eps
        dn[c] -= eps
        fd = (grid_loss(up) - grid_loss(dn)) / (2 * eps)
        gc = g[b, c].item()
        assert abs(fd - gc) <= 1e-6 * max(abs(gc), 1e-3 * gmax), (b, c, fd, gc)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_dehierarchize_fn_gradient(dtype, tol):
    """d/d alpha of <D alpha, w> is D^T w (the oracle's transpose)."""
    levels = (5, 4, 3)
    rng = np.random.default_rng(17)
    a = rng.uniform(-1, 1, inputs.num_points(levels))
    w = rng.uniform(-1, 1, a.size)
    alpha = torch.tensor(a, dtype=dtype, device="cuda", requires_grad=True)
    u = DehierarchizeFn.apply(alpha, levels)
    (u * torch.tensor(w, dtype=dtype, device="cuda")).sum().backward()
    ref = oracle.dehierarchize_adjoint(w, levels)
    assert np.abs(alpha.grad.double().cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    assert np.abs(u.detach().double().cpu().numpy() - oracle.dehierarchize(a, levels)).max() <= tol * 8
