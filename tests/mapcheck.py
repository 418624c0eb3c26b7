"""Comparison of a device map with the oracle's map, accepting differences only on the oracle's
ties (test helper).

The oracle decides every allocation and voxel update in FP64 and records the decisions that lie
within the single-precision rounding of their thresholds (oracle.OracleMap.alloc_tie,
brick_ties). The device decides in FP32, so its allocated (block, D) set and its voxels may
differ from the oracle's exactly there. The check is complete: every brick present on one side
only must be an allocation tie, and every voxel whose presence, sdf, weight or colour differs
beyond the value tolerances must carry the oracle's tie flag for that quantity. The number of
tie keys and tie voxels that actually differ is returned so that tests can report it.

Colour tolerance: the fused colour is the colour-weight average of the observed colours, so a
difference dW in the weights moves it by at most 255 dW / W. The weights are held to
w_rel W + w_abs; a common relative error cancels in the average, the absolute part does not, so
a voxel's colour is held to col_tol + 255 w_abs / W. This matters only where W is tiny (a voxel
seen only near the edge of a direction's angular zone, where the FP32 arc cosine of the direction
weight carries a relative error of 1e-3); the number of such voxels is returned.
"""
from __future__ import annotations

import numpy as np

# FP32 running averages against FP64 (units of tau; weights relative + absolute; colour 0..255)
SDF_TOL = 2e-4
W_REL = 1e-4
W_ABS = 1e-5
COL_TOL = 1e-2


def compare_maps(gm, om, sdf_tol=SDF_TOL, w_rel=W_REL, w_abs=W_ABS, col_tol=COL_TOL, chunk=8192):
    coords, vox = gm.export()
    gidx = {tuple(c): i for i, c in enumerate(coords)}
    okeys = set()
    out = dict(checked=0, bricks=0, tie_keys=0, tie_voxels=0, tie_colour=0, low_weight_colour=0)
    start = 0
    while True:
        oc, ov, ot = om.export(start, chunk)
        if len(oc) == 0:
            break
        start += len(oc)
        for c, o, t in zip(oc, ov, ot):
            key = tuple(int(x) for x in c)
            okeys.add(key)
            if key not in gidx:
                assert om.alloc_tie(*key) >= 0, ("brick only in the oracle, not a tie", key)
                out["tie_keys"] += 1
                continue
            g = vox[gidx[key]].astype(np.float64)
            tg, tc = (t & 1) > 0, (t & 2) > 0
            pg, po = g[:, 1] > 0, o[:, 1] > 0
            val = pg & po
            bad = pg != po
            bad[val] |= np.abs(g[val, 0] - o[val, 0]) > sdf_tol
            bad[val] |= np.abs(g[val, 1] - o[val, 1]) > w_rel * o[val, 1] + w_abs
            if np.any(bad & ~tg):
                i = np.nonzero(bad & ~tg)[0][:4]
                raise AssertionError(f"voxel differs without a tie: brick {key} voxels {i.tolist()} device "
                                     f"{g[i, :2].tolist()} oracle {o[i, :2].tolist()} ties {t[i].tolist()}")
            out["tie_voxels"] += int(np.sum(bad))
            cg, co = g[:, 5] > 0, o[:, 5] > 0
            cb = cg != co
            both = cg & co
            cdiff = np.abs(g[both, 2:5] - o[both, 2:5]).max(-1)
            cb[both] |= cdiff > col_tol + 255.0 * w_abs / o[both, 5]
            out["low_weight_colour"] += int(np.sum(cdiff > col_tol))
            cb[both] |= np.abs(g[both, 5] - o[both, 5]) > w_rel * o[both, 5] + w_abs
            if np.any(cb & ~(tc | tg)):
                i = np.nonzero(cb & ~(tc | tg))[0][:4]
                raise AssertionError(f"colour differs without a tie: brick {key} voxels {i.tolist()} device "
                                     f"{g[i, 2:].tolist()} oracle {o[i, 2:].tolist()} ties {t[i].tolist()}")
            out["tie_colour"] += int(np.sum(cb))
            out["checked"] += int(np.sum(val & ~tg))
            out["bricks"] += 1
    for key in set(gidx) - okeys:
        assert om.alloc_tie(*key) >= 0, ("brick only on the device, not a tie", key)
        out["tie_keys"] += 1
    return out
