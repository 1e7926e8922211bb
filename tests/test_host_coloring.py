"""The library's Welsh-Powell colouring (host code behind the C ABI; Sec. II.E) against the oracle,
colour for colour, and its argument checks.  CPU only: this entry point touches no device."""
import numpy as np
import pytest

import workloads as wl
from oracle import coloring as oco, neighbors as onb


@pytest.fixture(scope="module")
def api():
    from paper_1812_05264_gb300 import build, _lib
    build.build()
    _lib.load()
    from paper_1812_05264_gb300 import api as a
    return a


CASES = [
    ("chain r=2.5", lambda: (np.c_[2.5 * np.arange(6), np.zeros(6), np.zeros(6)], 2.5, None)),
    ("fcc 120, r=3.0", lambda: (wl.fcc_sphere(120, jitter=0.05, seed=3), 3.0, None)),
    ("fcc 500, r=6.0", lambda: (wl.fcc_sphere(500, jitter=0.05, seed=5), 6.0, None)),
    ("fcc 300, r=12.0", lambda: (wl.fcc_sphere(300, seed=7), 12.0, None)),
    ("fcc 40, r=100 (complete graph)", lambda: (wl.fcc_sphere(40, seed=1), 100.0, None)),
    ("fcc 60, r=1.0 (no edges)", lambda: (wl.fcc_sphere(60, seed=1), 1.0, None)),
    ("SC 6^3 periodic, r=1.0", lambda: (wl.sc_lattice(6)[0], 1.0, wl.sc_lattice(6)[1])),
    ("SC 8^3 periodic, r=2.0", lambda: (wl.sc_lattice(8)[0], 2.0, wl.sc_lattice(8)[1])),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_library_colouring_equals_the_oracle(api, name, make):
    pos, r, box = make()
    rp, col = onb.neighbor_csr(pos, r, box)               # self included, as the library builds it
    c, q = api.welsh_powell(rp, col)
    ref = oco.atom_colors(pos, r, box)
    assert np.array_equal(c, ref)
    assert q == int(ref.max()) + 1


def test_empty_and_single_vertex(api):
    c, q = api.welsh_powell(np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert c.size == 0 and q == 0
    c, q = api.welsh_powell(np.array([0, 1], np.int32), np.array([0], np.int32))
    assert c.tolist() == [0] and q == 1


@pytest.mark.parametrize("rp,col,what", [
    ([0, 2, 3], [0, 5, 1], "column index out of range"),
    ([0, 2, 1], [0, 1, 1], "row_ptr decreases"),
    ([0, 2, 3], [1, 0, 1], "columns not ascending"),
    ([0, 2, 3], [0, 1, 1], "one row only"),               # 0 lists 1, 1 does not list 0
    ([1, 2, 3], [0, 1, 1], "row_ptr[0]"),
])
def test_bad_graphs_are_rejected(api, rp, col, what):
    from paper_1812_05264_gb300 import _lib as L
    with pytest.raises(L.TbkError) as e:
        api.welsh_powell(np.array(rp, np.int32), np.array(col, np.int32))
    assert e.value.code == L.TBK_ERR_ARG and what in str(e.value)
