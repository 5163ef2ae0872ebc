"""Shared helpers of the test-suite: running the oracle on a workload and
comparing the CUDA path's outputs with it under the parity rules.

Parity rules (from the target tolerances of the rasterizer):
  * triangle ids equal on >= 99.99 % of valid pixels; a mismatch is allowed
    only where some edge distance |g| of either triangle is < 1e-6 or the
    relative depth gap of the two is < 1e-6;
  * coverage within 1e-5 absolute (the merge is order-free, so no pixel is
    exempt);
  * depth within 1e-5 relative where the ids agree.
"""
import numpy as np

import oracle

ID_FRAC = 0.9999
G_EPS = 1e-6
GAP_EPS = 1e-6
COV_TOL = 1e-5
DEPTH_TOL = 1e-5


def _dists(G, rec, t):
    r = rec[t]
    g = [G @ r[oracle.REC_N1:oracle.REC_N1 + 3], G @ r[oracle.REC_N2:oracle.REC_N2 + 3],
         G @ r[oracle.REC_N3:oracle.REC_N3 + 3]]
    depth = r[oracle.REC_D] / (G @ r[oracle.REC_N:oracle.REC_N + 3])
    return g, depth


def id_mismatch_allowed(G, rec, a, b):
    """Is a disagreement (oracle id a, CUDA id b) at direction G one the
    parity rule allows?"""
    gs, ds = [], []
    for t in (a, b):
        if t == oracle.NO_ID:
            continue
        g, d = _dists(G, rec, int(t))
        gs += g
        ds.append(d)
    if gs and min(abs(x) for x in gs) < G_EPS:
        return True
    if len(ds) == 2 and abs(ds[0] - ds[1]) <= GAP_EPS * abs(ds[0]):
        return True
    return False


def compare(map32, rec, exp, got, pixels=None):
    """exp: oracle outputs (flat over `pixels` or full frame); got: CUDA
    outputs as numpy (same shape as the frame).  Returns a report dict and
    asserts the parity rules."""
    H, W = map32.shape[:2]
    flat_map = map32.reshape(-1, 4).astype(np.float64)
    if pixels is None:
        pixels = np.arange(W * H)
    e_id = exp["id"].ravel()
    e_cov = exp["cov"].ravel()
    e_depth = exp["depth"].ravel()
    g_id = got["id"].reshape(-1)[pixels].astype(np.uint32)
    g_cov = got["cov"].reshape(-1)[pixels].astype(np.float64)
    g_depth = got["depth"].reshape(-1)[pixels].astype(np.float64)
    valid = flat_map[pixels, 3] > 0
    mism = np.nonzero((e_id != g_id) & valid)[0]
    bad = [q for q in mism if not id_mismatch_allowed(flat_map[pixels[q], :3], rec, e_id[q], g_id[q])]
    n_valid = int(valid.sum())
    rep = {
        "n_valid": n_valid,
        "id_mismatch": int(len(mism)),
        "id_mismatch_unexplained": len(bad),
        "id_equal_frac": 1.0 - len(mism) / max(1, n_valid),
        "cov_max_err": float(np.abs(e_cov - g_cov).max()) if len(e_cov) else 0.0,
    }
    same = (e_id == g_id) & (e_id != oracle.NO_ID)
    rep["depth_max_rel"] = float((np.abs(g_depth[same] / e_depth[same] - 1)).max()) if same.any() else 0.0
    assert (~valid <= (g_id == oracle.NO_ID)).all(), "invalid pixels must stay empty"
    assert np.all(g_cov[~valid] == 0.0)
    assert rep["id_equal_frac"] >= ID_FRAC, rep
    assert rep["id_mismatch_unexplained"] == 0, (rep, bad[:5])
    assert rep["cov_max_err"] <= COV_TOL, rep
    assert rep["depth_max_rel"] <= DEPTH_TOL, rep
    return rep
