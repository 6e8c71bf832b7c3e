"""Field checkpoints (raw float64 arrays behind a JSON header): a round trip keeps every bit, the
header describes the file, the arrays are 64-byte aligned, and damaged or foreign files are
refused."""
import json

import numpy as np
import pytest

from paper_1811_02605_gb300 import checkpoint as CK
from paper_1811_02605_gb300 import inputs as I


def _state(d, seed=5):
    rng = np.random.default_rng(seed)
    return {k: rng.normal(size=s) for k, s in CK.field_shapes(d.nr, d.nt, d.np).items()}


@pytest.mark.parametrize("d", [I.GridDesc(5, 6, 8, 1.0, 3.0, 1.1), I.GridDesc(9, 7, 10, 1.0, 6.0, 1.08)])
def test_round_trip_keeps_every_bit(tmp_path, d):
    st = _state(d)
    st["vr"][0, 0, 0] = np.nan   # any bit pattern survives
    st["bp"][1, 2, 3] = -0.0
    path = str(tmp_path / "c.mhd")
    h = CK.save(path, d, st, step=17, time=0.25, meta=dict(nu=1e-3, note="x"))
    h2, out = CK.load(path)
    assert h2 == json.loads(json.dumps(h))
    for k in CK.NAMES:
        assert out[k].shape == st[k].shape
        assert out[k].tobytes() == np.ascontiguousarray(st[k]).tobytes(), k
    assert h2["step"] == 17 and h2["time"] == 0.25 and h2["meta"]["nu"] == 1e-3
    assert h2["grid"] == dict(nr=d.nr, nt=d.nt, np=d.np, r0=d.r0, r1=d.r1, stretch=d.stretch)


def test_layout_header_line_and_alignment(tmp_path):
    d = I.GridDesc(4, 4, 8, 1.0, 2.0, 1.0)
    path = str(tmp_path / "c.mhd")
    h = CK.save(path, d, _state(d))
    raw = open(path, "rb").read()
    first = raw.split(b"\n", 1)[0]
    assert json.loads(first.decode())["format"] == "mhd-fields"
    offs = [a["offset"] for a in h["arrays"]]
    assert offs[0] == len(first) + 1 and all(o % 64 == 0 for o in offs)
    assert offs == sorted(offs) and [a["name"] for a in h["arrays"]] == list(CK.NAMES)
    a = h["arrays"][2]
    np.testing.assert_array_equal(np.frombuffer(raw[a["offset"]:a["offset"] + a["nbytes"]], "<f8"),
                                  _state(d)["bp"].ravel())
    assert len(raw) == h["arrays"][-1]["offset"] + h["arrays"][-1]["nbytes"]


def test_refuses_bad_input(tmp_path):
    d = I.GridDesc(4, 4, 8, 1.0, 2.0, 1.0)
    st = _state(d)
    with pytest.raises(ValueError):
        CK.save(str(tmp_path / "a"), d, {k: v for k, v in st.items() if k != "vp"})
    bad = dict(st, br=st["br"][:-1])
    with pytest.raises(ValueError):
        CK.save(str(tmp_path / "a"), d, bad)
    p = tmp_path / "junk"
    p.write_bytes(b"not a header\n" + b"\0" * 100)
    with pytest.raises(ValueError):
        CK.load(str(p))
    path = str(tmp_path / "c.mhd")
    CK.save(path, d, st)
    raw = open(path, "rb").read()
    (tmp_path / "cut").write_bytes(raw[:-8])   # truncated payload
    with pytest.raises(ValueError):
        CK.load(str(tmp_path / "cut"))
