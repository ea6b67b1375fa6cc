"""CPU-side checks of the C ABI: the library loads and exports what include/qst.h declares.

No compute call is made (there may be no GPU); only host-only entry points run.
"""
import os
import re

import pytest

from paper_2207_05341_gb300 import qst

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(qst_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(qst.LIB_PATH):
        from paper_2207_05341_gb300 import build
        build.build()
    return qst.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert "qst_init" in declared and "qst_step" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(qst.EXPORTED) <= declared


def test_host_only_entry_points(lib):
    o = qst.qst_default_options()
    assert o.lr == pytest.approx(1e-3) and o.eta_minus == 0.5 and o.eta_plus == 1.2
    assert o.step_min == 1e-6 and o.step_max == 50.0 and o.leaky_slope == 0.01
    assert o.mapping == qst.QST_MAP_CHOL_H and o.precision == qst.QST_FP32
    for N in (1, 2, 11, 12):
        n, H = 4 ** N, 2 * N
        assert qst.qst_theta_size(N) == 2 * H * n + n + H
    assert qst.qst_theta_size(0) == 0 and qst.qst_theta_size(13) == 0
    assert "invalid" in qst.strerror(qst.QST_E_INVAL)
    assert "clamp" in qst.strerror(qst.QST_W_CLAMP)


def test_binding_povm_matches_paper():
    import numpy as np
    import oracle as O
    flat = qst.tetrahedral_povm_flat().reshape(4, 2, 2, 2)
    np.testing.assert_allclose(flat[..., 0] + 1j * flat[..., 1], O.tetrahedral_povm(), atol=1e-16)


def test_rprop_bounds_are_checked_on_the_host(lib):
    """lr, step_min and step_max must lie in [2^-33, 2^30]: the Rprop state word then encodes the
    previous gradient sign exactly.  The check runs before any device call (no GPU needed here)."""
    for field, value in (("step_max", 2.0 ** 31), ("step_min", 2.0 ** -34), ("lr", 2.0 ** 31), ("lr", 1e-12)):
        o = qst.qst_default_options()
        setattr(o, field, value)
        with pytest.raises(qst.QstError) as e:
            qst.qst_init(3, opt=o)
        assert e.value.status == qst.QST_E_INVAL, (field, value)


def test_option_validation_before_any_device_call(lib):
    """Invalid combinations are refused by qst_init on the host, before it touches a device."""
    def status(N, **kw):
        o = qst.qst_default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        with pytest.raises(qst.QstError) as e:
            qst.qst_init(N, opt=o)
        return e.value.status
    assert status(2, network=qst.QST_NET_CNN) == qst.QST_E_INVAL  # 2^(N-3)-square pooling windows
    assert status(5, network=7) == qst.QST_E_INVAL
    assert status(8, mapping=qst.QST_MAP_CHOL_DELTA, precision=qst.QST_MIXED) == qst.QST_E_UNSUPPORTED
    assert status(6, mapping=qst.QST_MAP_ABS_P, precision=qst.QST_MIXED) == qst.QST_E_UNSUPPORTED
    assert status(4, mapping=qst.QST_MAP_ABS_P, P=0.0) == qst.QST_E_INVAL
    assert status(6, precision=qst.QST_MIXED) == qst.QST_E_UNSUPPORTED  # the tensor-core path starts at N = 7
    assert status(11, precision=qst.QST_FP64) == qst.QST_E_INVAL  # FP64 contexts stop at N = 10
    assert status(13) == qst.QST_E_INVAL
    assert status(4, mapping=9) == qst.QST_E_INVAL
    assert status(4, eta_plus=1.0) == qst.QST_E_INVAL
    assert status(8, mapping=qst.QST_MAP_ABS_P, precision=qst.QST_MIXED, eig_refine=2) == qst.QST_E_INVAL
    assert qst.qst_default_options().eig_refine == 1


def test_parameter_counts_of_both_networks(lib):
    for N in (3, 7, 11, 12):
        n, H = 4 ** N, 4 * N
        assert qst.qst_theta_size_net(N, qst.QST_NET_CNN) == H * n + n + H * 640 + H + 90 + 10
        assert qst.qst_theta_size_net(N, qst.QST_NET_FNN) == qst.qst_theta_size(N)
    assert qst.qst_theta_size_net(2, qst.QST_NET_CNN) == 0 and qst.qst_theta_size_net(13, qst.QST_NET_CNN) == 0


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without libqst.so the binding raises instead of computing anything elsewhere."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2207_05341_gb300 import qst\n"
            "try:\n    qst.load(%r)\nexcept RuntimeError as e:\n    print('raised', 'not found' in str(e))\n"
            % (ROOT, str(tmp_path / "libqst.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "raised True"


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/qst.h is a C ABI: it compiles as strict C99 and a C program links against libqst.so
    (only host-only entry points are called)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_qst.c"
    src.write_text('#include "qst.h"\n#include <stdio.h>\n'
                   "int main(void) {\n"
                   "  qst_options o;\n  qst_default_options(&o);\n"
                   '  printf("%zu %zu %d\\n", qst_theta_size(3), qst_theta_size_net(3, QST_NET_CNN), o.precision);\n'
                   "  return 0;\n}\n")
    exe = tmp_path / "use_qst"
    libdir = os.path.dirname(qst.LIB_PATH)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", f"-I{os.path.join(ROOT, 'include')}",
                        str(src), f"-L{libdir}", "-lqst", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    n3, H = 4 ** 3, 6
    assert out.stdout.split() == [str(2 * H * n3 + n3 + H), str(12 * n3 + n3 + 12 * 640 + 12 + 100), str(qst.QST_FP32)]


def test_static_probs_refuses_host_buffers_before_any_launch(lib):
    """qst_probs_static checks that rho and p are device memory before it launches anything: host
    buffers (or a machine without a GPU) give QST_E_INVAL, never a kernel fault."""
    import numpy as np
    rho = np.zeros((8, 8), dtype=np.complex64)
    p = np.zeros(64, dtype=np.float32)
    with pytest.raises(qst.QstError) as e:
        qst.qst_probs_static(3, rho, p)
    assert e.value.status == qst.QST_E_INVAL


def _tuned_defaults():
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2207_05341_gb300", "csrc", "tuned.h")).read()
    get = lambda name: int(re.search(r"constexpr int %s = (\d+);" % name, src).group(1))
    return {"bulk_chunks_per_cta": get("kTunedBulkChunksPerCta"), "fused_ctas_per_sm": get("kTunedFusedCtasPerSm"),
            "fused_max_qubits": get("kTunedFusedMaxQubits"), "batch_concurrent_runs": get("kTunedBatchConcurrentRuns")}


def test_tuning_defaults_and_validation(lib):
    """qst_get_tuning starts from the autotuner's table; qst_set_tuning refuses values out of range and
    leaves the others as they were (host only, no device call)."""
    start = qst.qst_get_tuning()
    assert start == _tuned_defaults()
    try:
        for bad in ({"bulk_chunks_per_cta": 0}, {"fused_ctas_per_sm": 3}, {"fused_ctas_per_sm": 0},
                    {"fused_max_qubits": 8}, {"fused_max_qubits": -1}, {"batch_concurrent_runs": 2}):
            with pytest.raises(qst.QstError) as e:
                qst.qst_set_tuning(**bad)
            assert e.value.status == qst.QST_E_INVAL
            assert qst.qst_get_tuning() == start
        qst.qst_set_tuning(bulk_chunks_per_cta=4, fused_max_qubits=0)
        assert qst.qst_get_tuning() == dict(start, bulk_chunks_per_cta=4, fused_max_qubits=0)
    finally:
        qst.qst_set_tuning(**start)


def test_autotuner_writes_its_choice(tmp_path, monkeypatch):
    from paper_2207_05341_gb300 import autotune
    pkg = tmp_path / "pkg"
    (pkg / "csrc").mkdir(parents=True)
    src = open(os.path.join(autotune.HERE, "csrc", "tuned.h")).read()
    (pkg / "csrc" / "tuned.h").write_text(src)
    monkeypatch.setattr(autotune, "HERE", str(pkg))
    log = tmp_path / "log.json"
    log.write_text('{"best": {"bulk_chunks_per_cta": 23, "fused_max_qubits": 5, "fused_ctas_per_sm": 1}}')
    autotune.main(["--apply", str(log)])
    out = (pkg / "csrc" / "tuned.h").read_text()
    assert "kTunedBulkChunksPerCta = 23;" in out and "kTunedFusedMaxQubits = 5;" in out
    assert "kTunedFusedCtasPerSm = 1;" in out and "kFusedThreads = 512;" in out
