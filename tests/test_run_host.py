"""The command-line front end (paper_2403_01039_gb300/run.py) on the host: atom-file
parsing and validation, the solute-centred grid, argument checks, and a loud failure when
no GPU is present (the solve itself runs only in the library's kernels)."""
import numpy as np
import pytest

from paper_2403_01039_gb300 import run


def test_read_atoms(tmp_path):
    f = tmp_path / "a.txt"
    f.write_text("# x y z q sigma eps\n0 0 0 -0.5 3.2 0.1\n\n1.5 0 0 0.5 2.5 0.05\n")
    xyz, q, s, e = run.read_atoms(str(f))
    assert xyz.shape == (2, 3) and np.allclose(q, [-0.5, 0.5]) and np.allclose(s, [3.2, 2.5])
    assert np.allclose(e, [0.1, 0.05]) and xyz[1, 0] == 1.5


@pytest.mark.parametrize("text,msg", [
    ("0 0 0 0 3.0\n", "expected"),
    ("0 0 0 0 3.0 x\n", "not a number"),
    ("0 0 0 0 -3.0 0.1\n", ">= 0"),
    ("0 0 nan 0 3.0 0.1\n", "non-finite"),
    ("# only a comment\n", "no atoms"),
])
def test_read_atoms_rejects(tmp_path, text, msg):
    f = tmp_path / "bad.txt"
    f.write_text(text)
    with pytest.raises(ValueError, match=msg):
        run.read_atoms(str(f))


def test_grid_is_centred_on_the_solute():
    xyz = np.array([[1.0, 2.0, 3.0], [3.0, 4.0, 5.0]])
    g = run.centred_grid(xyz, 64, 0.5)
    centre = np.array(g["origin"]) + 32 * 0.5
    assert g["n"] == (64, 64, 64) and np.allclose(centre, [2.0, 3.0, 4.0])


def test_arguments(tmp_path):
    a = run.parse(["atoms.txt"])
    assert (a.solvent, a.n, a.closure, a.tol, a.precision, a.fields) == ("water_nacl", 128, "kh", 1e-6, 32, ["g"])
    with pytest.raises(SystemExit):
        run.parse(["atoms.txt", "--n", "63"])
    with pytest.raises(SystemExit):
        run.parse(["atoms.txt", "--closure", "py"])


def test_fails_loudly_without_a_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("this host has a GPU")
    f = tmp_path / "a.txt"
    f.write_text("0 0 0 0 3.5 0.2\n")
    with pytest.raises(Exception):
        run.main([str(f), "--solvent", "water3", "--n", "32", "--out", str(tmp_path / "r.npz")])
    assert not (tmp_path / "r.npz").exists()
