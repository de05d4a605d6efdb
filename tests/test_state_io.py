"""On-disk state and the run record (host only)."""
import json

import numpy as np
import pytest
import torch

from paper_1803_01262_gb300 import state_io as S


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_state_round_trip(tmp_path, dtype):
    phi = np.random.default_rng(1).random((3, 4, 5)).astype(dtype)
    S.save_state(tmp_path / "s", torch.from_numpy(phi), step=120, t=0.75, eps=0.01, gamma=1.0, seed=7)
    back, h = S.load_state(tmp_path / "s")
    assert back.dtype == dtype and np.array_equal(back, phi)
    assert h["step"] == 120 and h["t"] == 0.75 and h["shape"] == [3, 4, 5]
    assert h["params"] == {"eps": 0.01, "gamma": 1.0, "seed": 7}


def test_state_refuses_mismatch(tmp_path):
    phi = np.zeros((2, 2, 2))
    S.save_state(tmp_path / "s", phi, step=0, t=0.0)
    with open(tmp_path / "s.bin", "ab") as f:     # a truncated or appended dump
        f.write(b"\0" * 8)
    with pytest.raises(ValueError):
        S.load_state(tmp_path / "s")
    with pytest.raises(ValueError):
        S.save_state(tmp_path / "t", np.zeros((2, 2)), step=0, t=0.0)
    with pytest.raises(ValueError):
        S.save_state(tmp_path / "t", np.zeros((2, 2, 2), np.int32), step=0, t=0.0)


def test_run_log(tmp_path):
    log = S.RunLog(tmp_path / "run.jsonl")
    st = {"mass": 2.0, "min": 0.0, "max": 1.0, "n_strict": 0, "n_tol": 0}
    log.record(0, 0.0, st)
    log.record(10, 0.1, dict(st, mass=2.0 + 2e-12, n_strict=3), gcells=1.5)
    lines = [json.loads(x) for x in open(tmp_path / "run.jsonl")]
    assert [r["step"] for r in lines] == [0, 10]
    assert lines[0]["mass_drift_rel"] == 0.0 and abs(lines[1]["mass_drift_rel"] - 1e-12) < 1e-15
    assert lines[1]["n_strict"] == 3 and lines[1]["gcells"] == 1.5


def test_state_refuses_data_from_another_save(tmp_path):
    """A process that died between renaming the new data and the new header leaves the new
    data under the old header, with the same byte count: the header's hash refuses it."""
    import shutil
    S.save_state(tmp_path / "s", np.zeros((2, 3, 4)), step=1, t=0.1)
    shutil.copy(tmp_path / "s.json", tmp_path / "old.json")
    S.save_state(tmp_path / "s", np.ones((2, 3, 4)), step=2, t=0.2)
    shutil.copy(tmp_path / "old.json", tmp_path / "s.json")
    with pytest.raises(ValueError, match="SHA-256"):
        S.load_state(tmp_path / "s")
