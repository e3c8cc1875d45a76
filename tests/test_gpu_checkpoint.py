"""Checkpoint / resume of the setup (mg_save / mg_load), host-side failure
injection, and bitwise-reproducible reruns.

No test here faults, traps or hangs the GPU: failures are made on the host
(a NaN in the right-hand side, a corrupted or mismatched file, calls out of
order) and must come back as status codes with the context still usable.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import lattice as lat
from gpu_helpers import oracle_fine, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)


def _ctx(gb, seed, nvec=(16, 16), U=None):
    if U is None:
        U = syn.gauge_field(DIMS, 0.4, 3)
    p = gb.default_params(dims=DIMS, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=list(nvec),
                          mass=-0.3, csw=1.0, nlevels=3, prec_fine=1, prec_coarse=1,
                          setup_sweeps=6, seed=seed)
    return gb.Multigrid(p, to_dev(U)), U


def _setup(gb, mg):
    for l in range(2):
        gb.mg_setup_nullvecs(mg.ctx, l, None)
        gb.mg_build_coarse(mg.ctx, l)


def _links(gb, mg, level):
    lv = mg.levels[level]
    out = torch.empty((lv["volume"], 9, lv["ndof"], lv["ndof"]), dtype=torch.complex128,
                      device="cuda")
    gb.mg_get_coarse_links(mg.ctx, level, out)
    return to_np(out)


def test_save_load_resumes_without_setup(gpu_lib, tmp_path):
    gb = gpu_lib
    path = tmp_path / "setup.gbmg"
    mg, U = _ctx(gb, 11)
    with pytest.raises(gb.MGError) as e:  # nothing to save yet
        gb.mg_save(mg.ctx, path)
    assert e.value.status == gb.MG_ERR_STATE
    _setup(gb, mg)
    gb.mg_save(mg.ctx, path)
    b = to_dev(syn.gaussian_field((lat.volume(DIMS), 12), 121))
    x1 = torch.zeros_like(b)
    st1 = gb.mg_gcr_solve(mg.ctx, x1, b, 1e-10, 300)
    links = [_links(gb, mg, l) for l in (1, 2)]
    mg.close()
    mg2, _ = _ctx(gb, 999, U=U)  # other seed: the loaded setup must win
    gb.mg_load(mg2.ctx, path)
    for l in (1, 2):
        assert np.array_equal(_links(gb, mg2, l), links[l - 1])
    x2 = torch.zeros_like(b)
    st2 = gb.mg_gcr_solve(mg2.ctx, x2, b, 1e-10, 300)
    assert st2["iters"] == st1["iters"]
    assert st2["true_residual"] <= 1e-10
    assert rel_l2(to_np(x2), to_np(x1)) < 1e-6
    mg2.close()


def test_load_rejects_mismatch_corruption_and_truncation(gpu_lib, tmp_path):
    gb = gpu_lib
    path = tmp_path / "setup.gbmg"
    mg, U = _ctx(gb, 12)
    _setup(gb, mg)
    gb.mg_save(mg.ctx, path)
    mg.close()
    raw = path.read_bytes()
    bad = bytearray(raw)
    bad[-100] ^= 0x40  # one flipped bit in the payload
    (tmp_path / "corrupt.gbmg").write_bytes(bytes(bad))
    (tmp_path / "short.gbmg").write_bytes(raw[:-1000])
    other, _ = _ctx(gb, 12, nvec=(8, 16), U=U)
    same, _ = _ctx(gb, 12, U=U)
    for ctx, f in ((other.ctx, path), (same.ctx, tmp_path / "corrupt.gbmg"),
                   (same.ctx, tmp_path / "short.gbmg"), (same.ctx, tmp_path / "missing")):
        with pytest.raises(gb.MGError) as e:
            gb.mg_load(ctx, f)
        assert e.value.status == gb.MG_ERR_ARG
    gb.mg_load(same.ctx, path)  # the intact file still loads afterwards
    other.close()
    same.close()


def test_nan_right_hand_side_is_reported_and_context_stays_usable(gpu_lib):
    gb = gpu_lib
    mg, U = _ctx(gb, 13)
    _setup(gb, mg)
    b = syn.gaussian_field((lat.volume(DIMS), 12), 122)
    bad = b.copy()
    bad[17, 3] = np.nan
    x = torch.zeros((lat.volume(DIMS), 12), dtype=torch.complex128, device="cuda")
    st = gb.mg_gcr_solve(mg.ctx, x, to_dev(bad), 1e-10, 50, check=False)
    assert st["status"] == gb.MG_ERR_NUMERICAL
    st = gb.mg_gcr_solve(mg.ctx, x, to_dev(b), 1e-10, 300)
    res = np.linalg.norm(b - oracle_fine(U, DIMS, -0.3).apply(to_np(x))) / np.linalg.norm(b)
    assert res <= 1.05e-10
    mg.close()


def test_reruns_are_bitwise_identical(gpu_lib):
    """Deterministic reductions (fixed grids, no atomics on data paths) and
    counter-based random starts: two contexts with the same seed give
    identical coarse operators, and every solve the same bits."""
    gb = gpu_lib
    b = to_dev(syn.gaussian_field((lat.volume(DIMS), 12), 123))
    runs = []
    for _ in range(2):
        mg, U = _ctx(gb, 14)
        _setup(gb, mg)
        x = torch.zeros_like(b)
        st = gb.mg_gcr_solve(mg.ctx, x, b, 1e-10, 300)
        xa = to_np(x)
        x.zero_()
        st_again = gb.mg_gcr_solve(mg.ctx, x, b, 1e-10, 300)
        assert np.array_equal(to_np(x), xa) and st_again["history"] == st["history"]
        runs.append((xa, _links(gb, mg, 1), st["history"]))
        mg.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
