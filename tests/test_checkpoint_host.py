"""Checkpoint file format on the host: header and population field round trip, and the rejection of
files that are not checkpoints (no GPU needed)."""
import os

import numpy as np
import pytest

from paper_2409_01076_gb300 import checkpoint as C


def _header(nx=7, ny=5):
    return {"nx": nx, "ny": ny, "tau": 0.6123, "u_lid": -0.07, "tau_s": 1.0, "bc": 0x85, "precision": 1,
            "layout": 1, "collision": 2, "t": 123456789012}


def test_round_trip_is_exact(tmp_path):
    f = np.random.Generator(np.random.PCG64(1)).normal(size=(9, 5, 7))
    p = str(tmp_path / "a.ckp")
    C.write_checkpoint(p, _header(), f)
    assert os.path.getsize(p) == 96 + 9 * 5 * 7 * 8
    hdr, g = C.read_checkpoint(p)
    assert hdr == dict(_header(), rounding=0)         # written without a rounding field: nearest
    assert np.array_equal(f, g)
    C.write_checkpoint(p, dict(_header(), rounding=1), f)
    assert C.read_checkpoint(p)[0]["rounding"] == 1


def test_rejects_other_files(tmp_path):
    p = str(tmp_path / "b.ckp")
    with open(p, "wb") as fh:
        fh.write(b"NOTACKPT" + bytes(200))
    with pytest.raises(ValueError, match="not an SmrtLBM checkpoint"):
        C.read_checkpoint(p)
    q = str(tmp_path / "c.ckp")
    C.write_checkpoint(q, _header(), np.zeros((9, 5, 7)))
    with open(q, "r+b") as fh:
        fh.truncate(96 + 100)
    with pytest.raises(ValueError, match="population values present"):
        C.read_checkpoint(q)
    with pytest.raises(ValueError, match="shape"):
        C.write_checkpoint(q, _header(), np.zeros((9, 7, 5)))
