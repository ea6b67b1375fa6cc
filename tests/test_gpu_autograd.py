"""The torch.autograd bridge: gradcheck in FP64, and torch's own Rprop on the library gradient
reproduces the fused in-library Rprop step."""
import numpy as np
import pytest

import oracle as O
from paper_2207_05341_gb300 import qst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    if not os.path.exists(qst.LIB_PATH):
        from paper_2207_05341_gb300 import build
        build.build()
    qst.load()


def _inputs(N, seed):
    M = O.tetrahedral_povm()
    rho = synth.ginibre_mixed(N, 2, 100 + seed)
    f = synth.frequencies(synth.multinomial_counts(O.born_probabilities(rho, M).real, 10**5, 200 + seed))
    return f, synth.init_theta(N, 300 + seed)


def test_gradcheck_fp64():
    from paper_2207_05341_gb300.autograd import QstLikelihood
    N = 2
    f, theta = _inputs(N, 1)
    opt = qst.qst_default_options()
    opt.precision = qst.QST_FP64
    h = qst.qst_init(N, opt=opt)
    try:
        th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
        fd = torch.tensor(f, dtype=torch.float64, device="cuda")
        assert torch.autograd.gradcheck(lambda t: QstLikelihood.apply(t, fd, h), (th,), eps=1e-6, atol=1e-7,
                                        rtol=1e-5)
    finally:
        qst.qst_destroy(h)


def test_torch_rprop_on_library_gradient_matches_fused_step():
    from paper_2207_05341_gb300.autograd import NNQST
    N = 4
    f, theta = _inputs(N, 2)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    th0 = torch.tensor(theta, dtype=torch.float32, device="cuda")
    model = NNQST(N, th0)
    try:
        opt = torch.optim.Rprop(model.parameters(), lr=1e-3, etas=(0.5, 1.2), step_sizes=(1e-6, 50))
        losses_a = []
        for _ in range(3):
            opt.zero_grad()
            L = model(fd)
            L.backward()
            opt.step()
            losses_a.append(float(L.detach()))
        ctx = qst.qst_init(N)
        try:
            qst.qst_set_params(ctx, th0)
            losses_b = [qst.qst_step(ctx, fd)[0] for _ in range(3)]
            tb = torch.empty_like(th0)
            qst.qst_get_params(ctx, tb)
        finally:
            qst.qst_destroy(ctx)
        np.testing.assert_allclose(losses_a, losses_b, rtol=1e-6)
        diff = (model.theta.detach() - tb).abs()
        # the two Rprop implementations take the same sign decisions except on gradients at rounding level
        assert (diff > 1e-6).float().mean().item() < 1e-3
    finally:
        model.close()
