"""The synthetic workloads carry the geometry and sizes the paper prints
(tests/golden/paper_constants.json, each block cited)."""
import json
import os

import numpy as np

from synth import paper_workload

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_paper_scale_workload_matches_table_one_and_protocol():
    wl = paper_workload(p=660)
    pg, xp, md = GOLD["patient_geometry"], GOLD["xcat_protocol"], GOLD["model"]
    g = wl.grid
    assert [g.nx, g.ny, g.nz] == pg["volume_voxels"]
    assert [g.vx, g.vy, g.vz] == pg["voxel_mm"]
    assert (wl.det.nu, wl.det.nv) == (pg["projection_width_px"], pg["projection_height_px"])
    assert wl.p == xp["projections"]
    src = wl.views[:, 0:3]
    det = wl.views[:, 3:6]
    np.testing.assert_allclose(np.linalg.norm(src, axis=1), pg["sad_mm"], rtol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(src - det, axis=1), pg["sdd_mm"], rtol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(wl.views[:, 6:9], axis=1), pg["pixel_mm"], rtol=1e-12)
    ang = np.unwrap(np.arctan2(src[:, 1], src[:, 0]))
    assert np.degrees(ang[-1] - ang[0]) * xp["projections"] / (xp["projections"] - 1) == \
        np.float64(xp["arc_deg"]) or abs(np.degrees(ang[-1] - ang[0]) - 360 * 659 / 660) < 1e-9
    assert wl.ref.g == md["reference_gaussians_patients"]
    assert wl.levels == md["mbc_levels"]
    assert wl.coeff.shape[1] * wl.coeff.shape[2] == md["coefficients_per_projection"]
    # 11 frames/s over 60 s
    assert abs(xp["projections"] / xp["frame_rate_fps"] - xp["scan_s"]) < 1.0
