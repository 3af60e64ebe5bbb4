"""Host logic of bench.py that needs no GPU: the code hash that ties stored ncu traffic to
the kernels it measured (comments do not count, code does), and the workload record."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _copy_tree(tmp_path):
    dst = tmp_path / "paper_1504_07499_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_1504_07499_gb300", "csrc"), dst)
    return dst


def test_code_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    base = bench._kernel_sha()
    csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._kernel_sha() == base
    f = csrc / "hmg_fast.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n/* and a block\n   comment */\n" + text.replace("\n", "  // tail\n", 3))
    assert bench._kernel_sha() == base
    f.write_text(text.replace("constexpr int fx_rows() { return 128 /", "constexpr int fx_rows() { return 256 /", 1))
    assert bench._kernel_sha() != base


def test_workload_record():
    cfg = bench.workload_config("fp32bulk")
    assert cfg["N"] == bench.N_GRID == 256 and cfg["workload"].startswith("rsa256")
    assert cfg["k"] == list(bench.K_PHASES) and cfg["tol"] == 1e-8


def test_torch_fft_comparison_sweep_matches_the_oracle():
    """The cuFFT comparison leg's sweep, run here on the CPU, against one oracle sweep."""
    import numpy as np
    import pytest
    torch = pytest.importorskip("torch")
    from oracle import em as om
    from paper_1504_07499_gb300 import inputs as I
    N, k = 16, I.K_PHASES
    ph = om.voxelize(I.generate_spheres(7, 10, 0.3).spheres, 0.3, N)
    k0 = om.reference_k0(k)
    for E in ((1.0, 0.0, 0.0), (0.0, 0.0, 1.0)):
        ref = om.em_solve(ph, k, E, tol=0.0, max_iter=1, record=True)
        sweep = bench.torch_fft_sweep(torch.from_numpy(ph.reshape(-1)), k, N, "cpu")
        kp = torch.tensor(np.asarray(k) + k0, dtype=torch.float32)[torch.from_numpy(ph).long()]
        tau0 = kp[None] * torch.tensor(E, dtype=torch.float32)[:, None, None, None]
        e1 = (sweep(tau0, E) / kp[None]).double().numpy()
        assert np.abs(e1 - ref.e).max() < 1e-5 * np.abs(ref.e).max()
