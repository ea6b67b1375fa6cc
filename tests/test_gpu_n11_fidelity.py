"""Reconstruction fidelity at N = 11 on the GPU against the FP64 oracle's.

Workload and stored oracle values: tests/golden/make_n11_fidelity.py (noise-free probabilities of a
Haar pure state, the Fig. 2-4 setting of Sec. 4), whose output n11_reconstruction_fidelity.txt holds
<psi| rho^ |psi> of the oracle after 20 and 50 Rprop iterations.  The library runs the same
iterations from the same float32 parameters and f; its state fidelity must agree within 1e-4
(mixed FP16x3 / BF16x3 tensor-core products, and the plain FP32 path).  The fidelity of the
library's rho^ (complex64) is evaluated in complex128 on the host.
"""
import importlib.util
import os

import numpy as np
import pytest

from paper_2207_05341_gb300 import qst

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    spec = importlib.util.spec_from_file_location("make_n11_fidelity", os.path.join(HERE, "golden",
                                                                                   "make_n11_fidelity.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(qst.LIB_PATH):
        from paper_2207_05341_gb300 import build
        build.build()
    qst.load()


@pytest.fixture(scope="module")
def workload():
    G = _golden()
    psi, f, theta = G.inputs()
    return G, psi, f, theta, G.read()


@pytest.mark.parametrize("prec", [qst.QST_MIXED, qst.QST_MIXED_BF16, qst.QST_FP32])
def test_n11_reconstruction_fidelity_matches_oracle(workload, prec):
    G, psi, f, theta, want = workload
    N, d = G.N, 1 << G.N
    opt = qst.qst_default_options()
    opt.precision = prec
    ctx = qst.qst_init(N, opt=opt)
    try:
        qst.qst_set_params(ctx, theta)
        f_dev = torch.from_numpy(f).cuda()
        rho = torch.empty((d, d), dtype=torch.complex64, device="cuda")
        done = 0
        for k in sorted(want):
            qst.qst_reconstruct(ctx, f_dev, k - done, rho)
            done = k
            r = rho.cpu().numpy().astype(np.complex128)
            F = float(np.real(np.vdot(psi, r @ psi)))
            assert abs(F - want[k]) < 1e-4, (k, F, want[k])
        assert want[max(want)] > 0.99
    finally:
        qst.qst_destroy(ctx)
