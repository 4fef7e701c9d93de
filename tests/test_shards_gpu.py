"""Logical shards on one GPU: variables never interact, so a wide CFG
split into word ranges (each range analysed as a CFG of its own, as a
multi-GPU run would place them) gives, range by range, exactly the full
analysis's states, access flags and transfers."""
import numpy as np
import pytest

from paper_2406_13881_b300 import _native, workload as wl

pytestmark = pytest.mark.gpu


def _xfers(r, w_off=0):
    x = r["edge_xfers"]
    return sorted(zip(x["edge"].tolist(), (x["word"] + w_off).tolist(), x["to_bits"].tolist(),
                      x["from_bits"].tolist()))


@pytest.mark.parametrize("cuts", [(0, 2, 5), (0, 1, 3, 4, 5)])
def test_word_range_shards_equal_full(cuts):
    rng = np.random.default_rng(31)
    g = wl.structured(4100, 6000, 300, acc_min=1, acc_max=10, var_dist="zipf")  # 5 words
    g.entry_dev_valid = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
    g.exit_host_live = rng.integers(0, 2**63, size=g.W, dtype=np.uint64)
    full = _native.analyze(g, keep_states=True)
    got = []
    flags = np.zeros_like(full["acc_flag"])
    for w0, w1 in zip(cuts[:-1], cuts[1:]):
        sub, keep = wl.restrict_words(g, w0, w1)
        r = _native.analyze(sub, keep_states=True)
        for k in ("h_in", "d_in", "h_out", "d_out", "live_in"):
            np.testing.assert_array_equal(r[k], full[k][:, w0:w1], err_msg=k)
        np.testing.assert_array_equal(r["from_exit"], full["from_exit"][:, w0:w1])
        flags[keep] = r["acc_flag"]
        got += _xfers(r, w0)
    np.testing.assert_array_equal(flags, full["acc_flag"])
    assert sorted(got) == _xfers(full)
