"""Helpers that put library results and oracle results side by side."""
import numpy as np


def dense_edges(res, n_edges, W):
    """Dense [E, W] to/from planes from the library's sparse edge records;
    asserts that no (edge, word) appears twice."""
    to = np.zeros((n_edges, W), dtype=np.uint64)
    fr = np.zeros((n_edges, W), dtype=np.uint64)
    x = res["edge_xfers"]
    if len(x):
        key = x["edge"].astype(np.int64) * W + x["word"]
        assert len(np.unique(key)) == len(key), "duplicate edge transfer records"
        assert ((x["to_bits"] | x["from_bits"]) != 0).all(), "empty transfer record"
        to[x["edge"], x["word"]] = x["to_bits"]
        fr[x["edge"], x["word"]] = x["from_bits"]
    return to, fr


def assert_matches_oracle(g, res, orc, words=None, acc_keep=None):
    """Bit-exact comparison of every output (optionally restricted to the
    word columns ``words`` of the library result, against an oracle run on
    the same columns; ``acc_keep`` = library access indices the oracle saw)."""
    W = g.W
    cols = slice(None) if words is None else words
    np.testing.assert_array_equal(res["h_in"][:, cols], orc["h_in"], err_msg="h_in")
    np.testing.assert_array_equal(res["d_in"][:, cols], orc["d_in"], err_msg="d_in")
    if "h_out" in res:
        np.testing.assert_array_equal(res["h_out"][:, cols], orc["h_out"], err_msg="h_out")
        np.testing.assert_array_equal(res["d_out"][:, cols], orc["d_out"], err_msg="d_out")
    if "live_in" in res:
        np.testing.assert_array_equal(res["live_in"][:, cols], orc["live_in"], err_msg="live_in")
    flags = res["acc_flag"] if acc_keep is None else res["acc_flag"][acc_keep]
    np.testing.assert_array_equal(flags, orc["acc_flag"], err_msg="acc_flag")
    to, fr = dense_edges(res, g.n_edges, res["h_in"].shape[1])
    np.testing.assert_array_equal(to[:, cols], orc["to_edge"], err_msg="to_edge")
    np.testing.assert_array_equal(fr[:, cols], orc["from_edge"], err_msg="from_edge")
    fx = orc["from_exit"]
    ex = res["exit_blocks"]
    np.testing.assert_array_equal(res["from_exit"][:, cols], fx[ex], err_msg="from_exit")
    others = np.ones(g.n_blocks, dtype=bool)
    others[ex] = False
    assert not fx[others].any(), "oracle exit transfer at a block the library does not list"
    if "call_to" in orc and len(orc["call_to"]):
        sites = np.flatnonzero(np.asarray(g.acc, dtype=np.uint32) >> np.uint32(31))
        np.testing.assert_array_equal(res["call_site_acc"], sites, err_msg="call_site_acc")
        for k in ("call_to", "call_from", "call_entry_h", "call_entry_d", "call_exit_live"):
            np.testing.assert_array_equal(res[k][:, cols], orc[k], err_msg=k)
