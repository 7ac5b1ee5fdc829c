"""Host-side helpers of bench.py that feed its JSON line (no GPU): the default step counts,
the measured-peak lookup, the ncu traffic record keyed by the kernel source, the measured
host core count of the oracle baseline, and the cuFFT comparison failing soft."""
import json
import os
import sys

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_defaults_meet_the_timing_rules(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"
    assert a.workload == "globule2000_256" and a.tol == 1e-6 and a.precision == 32


def test_peak_lookup(bench):
    peak, src = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert peak == float(json.load(open(path))["hbm_gbs"]) and src.startswith("measured")
    else:
        assert peak == 6800.0 and src.startswith("fallback")


def test_traffic_record_is_keyed_by_the_kernel_source(bench, tmp_path, monkeypatch):
    """A traffic figure taken on other kernel source reads as None (reported as null)."""
    rec = {"solute50_128": {"plane_fwd": {"kernels_sha": "0" * 16, "dram_bytes_per_launch": 1.0}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    csrc = tmp_path / "paper_2403_01039_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "rism3d_kernels.cuh").write_text("// other source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("plane_fwd", "solute50_128") is None
    assert bench.ncu_traffic("pencil", "solute50_128") is None
    import hashlib
    rec["solute50_128"]["plane_fwd"]["kernels_sha"] = hashlib.sha256(b"// other source\n").hexdigest()[:16]
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("plane_fwd", "solute50_128") == 1.0


def test_host_core_count_is_measured(bench):
    class C:
        def __init__(self, wall, cpu):
            self.wall, self.cpu = wall, cpu
    assert bench._cores_used(C(10.0, 10.2))[0] == 1
    assert bench._cores_used(C(2.0, 15.4), C(2.0, 15.0))[0] == 8
    with bench._HostClock() as hc:
        sum(i * i for i in range(200000))
    assert hc.wall > 0.0 and hc.cpu >= 0.0


def test_cufft_comparison_fails_soft(bench):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("the soft failure is for hosts without a GPU")
    r = bench.cufft_comparison(3, (8, 8, 8), 32, 0.1)
    assert set(r) == {"error"}


def test_oracle_sample_scales_the_atom_sums(bench):
    """The bounded CPU sample builds the oracle's Problem from a few atoms and scales the
    atom-dependent sums to the whole solute: the estimate must lie between the subset's cost
    and the subset's cost times n / a."""
    from paper_2403_01039_gb300 import synth
    solv = synth.water_3site()
    chi = np.load(os.path.join(bench.ROOT, "tests", "golden", "chi_water3.npz"))
    solv.update(chi=chi["chi"], dk=float(chi["dk"]))
    grid = synth.cubic_grid(16, 0.5)
    sol = synth.random_solute(12, 4.0, 5)
    t_setup, t_iter, clocks, how = bench.oracle_sample(solv, grid, sol, "kh", 3, 5, 2, 3)
    assert t_iter > 0 and len(clocks) == 3 and "3 of 12 atoms" in how
    assert clocks[0].wall <= t_setup <= clocks[0].wall * 4 + clocks[1].wall * 4
