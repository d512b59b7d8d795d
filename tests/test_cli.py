"""The command line (python -m paper_2604_06602_gb300): input checks on the
host, and a detrend of a small CSR file on the GPU against the oracle."""
import json

import numpy as np
import pytest

import oracle
from paper_2604_06602_gb300 import __main__ as cli
from paper_2604_06602_gb300 import synth
from tests.helpers import compare_detr, compare_trend


def test_npy_input_needs_a_window(tmp_path):
    f = tmp_path / "x.npy"
    np.save(f, np.ones(100, np.float32))
    with pytest.raises(SystemExit):
        cli.main(["detrend", str(f), str(tmp_path / "o.npz")])


def test_window_count_must_match_curves(tmp_path):
    f = tmp_path / "x.npz"
    np.savez(f, flux=np.ones(10, np.float32), offsets=np.array([0, 4, 10]), W=np.array([3], np.int32))
    with pytest.raises(SystemExit):
        cli.main(["detrend", str(f), str(tmp_path / "o.npz")])


@pytest.mark.gpu
def test_detrend_file_matches_oracle(tmp_path, capsys):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    xs = [synth.random_curve(31, 3000, nan_runs=1), synth.random_curve(32, 800)]
    flux = np.concatenate(xs).astype(np.float32)
    off = np.array([0, 3000, 3800], np.int64)
    cad = np.array([synth.CADENCE_TESS_2MIN, synth.CADENCE_KEPLER_LC])
    src, dst = tmp_path / "in.npz", tmp_path / "out.npz"
    np.savez(src, flux=flux, offsets=off, cadence=cad)
    assert cli.main(["detrend", str(src), str(dst)]) == 0
    info = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert info == {"curves": 2, "samples": 3800, "windows": [25, 361]}
    z = np.load(dst)
    for k, (x, W) in enumerate(zip(xs, (361, 25))):
        ref = oracle.detrend(x, W)
        s = slice(off[k], off[k + 1])
        compare_trend(z["trend"][s], ref["trend"], what="cli curve %d" % k)
        compare_detr(z["detr"][s], ref["detr"], what="cli curve %d" % k)
    assert cli.main(["plan", "361", "12500"]) == 0
    plan = json.loads(capsys.readouterr().out.strip())
    assert plan["lanes"] * plan["slots"] >= 361
