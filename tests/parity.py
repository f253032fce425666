"""Comparison of GPU hits with the oracle under the stated tolerances: identical hit/miss and patch id
on every ray the oracle does not flag (silhouette or near tie), t within 1e-4 relative, u and v within
one leaf cell (2^-L)."""
import numpy as np

MISS = 0xFFFFFFFF
REL_T = 1e-4


def compare(g, o, L, rel_t=REL_T, max_flagged_frac=0.02, require_all=True):
    flags = o["flags"]
    ok = flags == 0
    n = len(ok)
    ghit = g["pid"] != MISS
    ohit = o["pid"] != MISS
    bad_hm = ok & (ghit != ohit)
    bad_pid = ok & ohit & ghit & (g["pid"] != o["pid"])
    both = ok & ohit & ghit & (g["pid"] == o["pid"])
    tt = o["t"][both]
    bad_t = np.abs(g["t"][both].astype(np.float64) - tt) > rel_t * np.abs(tt)
    cell = 2.0 ** -L * (1 + 1e-6)
    bad_u = np.abs(g["u"][both].astype(np.float64) - o["u"][both]) > cell
    bad_v = np.abs(g["v"][both].astype(np.float64) - o["v"][both]) > cell
    # misses must be written as the documented miss record
    gmiss = ~ghit
    bad_miss = gmiss & ~(np.isinf(g["t"]) & (g["u"] == 0) & (g["v"] == 0))
    rep = dict(n=n, hits=int(ohit.sum()), flagged=int((~ok).sum()), bad_hitmiss=int(bad_hm.sum()),
               bad_pid=int(bad_pid.sum()), bad_t=int(bad_t.sum()), bad_u=int(bad_u.sum()), bad_v=int(bad_v.sum()),
               bad_miss_record=int(bad_miss.sum()),
               # flagged by each bit of the oracle's error model (bit 4, the silhouette test of moving the
               # origin by 1e-4 of the scene, only when the oracle ran with flags=2), and the rays that the
               # silhouette test alone flags: excluded by that rule although FP32 cannot change their answer
               flagged_by_bit=[int(((flags >> b) & 1).sum()) for b in range(5)],
               silhouette_only=int((flags == 16).sum()), flagged_fp32=int(((flags & 15) != 0).sum()))
    if require_all:
        assert rep["bad_hitmiss"] == 0 and rep["bad_pid"] == 0, rep
        assert rep["bad_t"] == 0 and rep["bad_u"] == 0 and rep["bad_v"] == 0, rep
        assert rep["bad_miss_record"] == 0, rep
        # the cap is on the FP32 error model (bits 0..3); the silhouette rule's exclusions are the rule's
        assert rep["flagged_fp32"] <= max_flagged_frac * max(n, 1) + 2, rep
    return rep
