"""CUDA path vs the FP64 oracle, through the C ABI (needs a B300).

Bit-exact: tile rectangles, depth keys, tiles touched, tile offsets, sorted
per-tile lists.  Floating point (see tests/parity.py): all 13 moment sums of
every (view, Gaussian) record within 1e-4 of the bound on their terms'
magnitudes; per-view new means 1e-3 px and new 2D covariances 1e-3 relative;
positions 1e-4 of the scene extent, rotations 1e-3 rad (the fitted covariance
within 2e-4 relative where two fitted eigenvalues are within 1e-3 of each
other), scales 1e-4 relative; rendered colour and transmittance 1e-4.  Pixel
counts may differ only by blend decisions the oracle recorded as lying inside
the FP32 window.  A quantity that the FP64 oracle itself cannot pin to half its
tolerance under FP32-sized perturbations is held to tol + K x that movement
instead (no solved Gaussian goes unchecked), and the share of such quantities
is capped per scene.
"""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
import synth
from tests import parity as P

pytestmark = pytest.mark.gpu

POS_TOL, ROT_TOL, SCALE_TOL, PIX_TOL = 1e-4, 1e-3, 1e-4, 1e-4
MU_TOL_PX, COV_TOL_REL = 1e-3, 1e-3
# moment sums: within this fraction of the bound on the sum of the terms'
# magnitudes (the FP32 weight and summation errors are relative to that sum)
MOM_TOL_REL = 1e-4
# Excluded shares.  A quantity is excluded from its flat tolerance when the FP64
# oracle itself moves by more than half of it under FP32-sized perturbations (or
# its status is unstable under them); it is then held to tol + K x that
# movement (K = 4; the largest GPU error measured on an excluded quantity was
# 2.5 x the oracle's movement).  The shares are properties of the seeded scenes
# and the oracle alone (no GPU input).  Measured: positions 0-3 per scene (at
# most 0.016 %); rotations none; scales 0.1 % (tiny), 0.8 % (ragged), 0 (32
# views), 10.7 % (capture_sub, 4 views), 9.6 % (the 5-view 320 x 240 batch
# frame), 2 of 59 .. 4 of 59 (full capture sample).  The caps add a margin.  The
# scale share of the few-view scenes is the thin axis of elongated Gaussians
# fitted from 3-5 views: the covariance system is weakly constrained there.
EXCL_CAPS = {
    "default": dict(pos=0.001, scale=0.02, angle=0.005, cov=0.05),
    "few_views": dict(pos=0.001, scale=0.13, angle=0.005, cov=0.05),
    "full_capture": dict(pos=0.001, scale=0.12, angle=0.005, cov=0.05),
}
EXCL_CAPS["capture_sub"] = EXCL_CAPS["few_views"]


def caps_for(scene):
    """Capture-preset scenes seen in at most 8 views get the few-view caps."""
    return EXCL_CAPS["few_views" if scene.name == "capture" and scene.num_views <= 8 else "default"]
# (view, Gaussian) records whose per-view decision lies within 5 % of a Sec. 5.1
# threshold or that hold a pixel with a blend decision inside the FP32 window
VIEW_MARGIN_CAP = 0.06
# pixels with a blend decision inside the FP32 window (the contract's 0.1 %)
RENDER_WINDOW_CAP = 0.001


@pytest.fixture(scope="module")
def gpu_ready():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02586_b300 import build as tbuild
    tbuild.build()
    return True


SCENES = {
    "tiny": lambda: synth.make_scene("tiny", 1),
    "capture_sub": lambda: synth.make_scene("capture", 3, n=20000, views=4),
    "ragged": lambda: synth.make_scene("tiny", 9, n=800, views=3, width=100, height=70, focal=80.0),
}
_cache = {}


def case(name):
    if name not in _cache:
        s = SCENES[name]()
        o = oracle.fit_motion(s)
        _cache[name] = (s, P.run_gpu(s), o, P.sensitivity(s, o))
    return _cache[name]


def near(x, thr):
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.abs(np.log(np.maximum(x, 1e-300) / thr)) < math.log(1.05)


def view_margins(orc):
    """(v, g) whose per-view decision lies near a threshold in the oracle."""
    M = orc["moments"]
    sw = M[..., 5]
    with np.errstate(divide="ignore", invalid="ignore"):
        mx, my = M[..., 2] / sw, M[..., 4] / sw
        cxx = M[..., 0] / sw - mx * mx
        cxy = M[..., 1] / sw - mx * my
        cyy = M[..., 3] / sw - my * my
        tr, dt = cxx + cyy, cxx * cyy - cxy * cxy
        lmin = 0.5 * (tr - np.sqrt(np.maximum(tr * tr - 4 * dt, 0)))
        det = sw ** 3 * dt
    return near(sw, 1e-3) | near(det, 1e-12) | near(lmin, 1e-4) | (M[..., 15] > 0.02 * sw) | (M[..., 16] > 0)


@pytest.mark.parametrize("name", list(SCENES))
def test_keys_bit_exact(gpu_ready, name):
    s, g, _, _ = case(name)
    k = oracle.keys(s)
    assert np.array_equal(g["rect"].astype(np.int32), k["rect"])
    assert np.array_equal(g["depth"], k["depth_bits"])
    assert np.array_equal(g["touched"], k["tiles_touched"])


@pytest.mark.parametrize("name", list(SCENES))
def test_bins_bit_exact(gpu_ready, name):
    s, g, _, _ = case(name)
    off, ent = oracle.bin_lists(s)
    assert int(g["counts"][0]) == len(ent) and int(g["counts"][3]) == 0
    assert np.array_equal(g["tile_off"].astype(np.int64), off)
    assert np.array_equal(g["pairs"], ent)


@pytest.mark.parametrize("scale", [1.0, 0.3])
def test_all_list_lengths_bin_bit_exact(gpu_ready, scale):
    """Dense 512x512 scenes whose tile lists span every sort path: the one-warp
    register sorts (2..512 keys), the shared-memory sort (..4096) and the
    run merge (longer)."""
    s = synth.make_scene("tiny", 3, n=20000, views=2, width=512, height=512, focal=512.0)
    s.means_opacity[:, :3] *= scale
    g = P.run_gpu(s)
    off, ent = oracle.bin_lists(s)
    d = np.diff(off)
    if scale == 1.0:
        assert all(((d > a) & (d <= b)).any() for a, b in
                   ((1, 32), (32, 64), (64, 128), (128, 256), (256, 512), (512, 1024), (1024, 4096)))
    else:
        assert d.max() > 4096
    assert int(g["counts"][0]) == len(ent) and int(g["counts"][3]) == 0
    assert np.array_equal(g["tile_off"].astype(np.int64), off)
    assert np.array_equal(g["pairs"], ent)


@pytest.mark.parametrize("dup", ["some", "all"])
def test_equal_depths_bin_bit_exact(gpu_ready, dup):
    """Copies of Gaussians have bit-equal depths, so their tile lists hold keys of
    one depth that only the Gaussian index orders (R18): lists of every sort path,
    with and without such keys, equal the oracle's."""
    import dataclasses
    s0 = synth.make_scene("tiny", 3, n=20000, views=2, width=512, height=512, focal=512.0)
    idx = (np.random.default_rng(5).choice(s0.n, 1500, replace=False) if dup == "some"
           else np.arange(s0.n))
    cat = lambda a: np.ascontiguousarray(np.concatenate([a, a[idx]]))
    s = dataclasses.replace(s0, means_opacity=cat(s0.means_opacity), quats=cat(s0.quats),
                            scales=cat(s0.scales), sh=cat(s0.sh), labels=cat(s0.labels))
    g = P.run_gpu(s)
    off, ent = oracle.bin_lists(s)
    assert int(g["counts"][0]) == len(ent) and int(g["counts"][3]) == 0
    assert np.array_equal(g["tile_off"].astype(np.int64), off)
    assert np.array_equal(g["pairs"], ent)
    # lists with and without equal depths, among the warp-sorted lengths
    hi = (ent >> np.uint64(32)).astype(np.int64)
    same = np.zeros(len(ent), bool)
    same[1:] = hi[1:] == hi[:-1]
    same[off[:-1][off[:-1] < len(ent)]] = False          # a list's first key has no predecessor in it
    tied = np.add.reduceat(same.astype(np.int64), off[:-1].clip(max=len(ent) - 1)) > 0
    n = np.diff(off)
    short = (n > 1) & (n <= 512)
    assert (tied & short).any()
    if dup == "some":
        assert (~tied & short).any()


def check_moments(s, o, g, tag=None, tile=(16, 16)):
    """All 13 moment sums and both pixel counts of every (view, Gaussian) record
    against the oracle's record restated in the library's frame.

    Each sum must lie within MOM_TOL_REL of the bound on the sum of its terms'
    magnitudes, plus what the FP32 pixel coordinates' absolute error eps allows:
    the library takes coordinates relative to the Gaussian's tile rectangle, so
    eps is a few units in the last place of |mu_2D - rectangle corner| +
    |origin shift|, and a sum with a coordinate factor x~_i moves by eps_i times
    the sum of its other factor's magnitudes.  Where the oracle recorded blend
    decisions inside the FP32 window (alpha vs 1/255, T (1 - alpha) vs 1e-4),
    each such decision taken differently moves a pixel count by one and a sum by
    at most that pixel's weight change (<= its weight, or 0.01 for a flipped
    contribution) times the largest feature value the Gaussian can reach."""
    lf = P.library_frame(s, o)
    L, mag = lf["mom"], lf["mag"]
    gm = g["view_moments"].astype(np.float64)
    pw, pc = o["moments"][..., 15], o["moments"][..., 16]
    assert np.all(np.abs(gm[..., 13] - L[..., 13]) <= pc)
    assert np.all(np.abs(gm[..., 14] - L[..., 14]) <= pc)
    rect = oracle.keys(s, tile=tile)["rect"].astype(np.float64)
    corner = np.stack([rect[..., 0] * tile[0], rect[..., 1] * tile[1]], -1)
    span = np.abs(o["mean2d"] - corner) + np.abs(lf["dl"])
    eps = 4 * 2.0 ** -24 * np.maximum(span, float(max(tile)))        # [V, n, 2]
    sw = L[..., 0]
    # the FP64 restatement itself rounds terms of size |oracle sums| + sw |r| |dl|
    big = np.abs(o["moments"][..., :12]).max(-1) + sw * (1 + np.abs(lf["r"]).sum(-1)) * \
        (1 + np.abs(lf["dl"]).sum(-1))
    bound = MOM_TOL_REL * mag + 1e-12 * big[..., None]
    bound[..., 1] += eps[..., 0] * sw
    bound[..., 2] += eps[..., 1] * sw
    bound[..., 3] += 2 * eps[..., 0] * mag[..., 1]
    bound[..., 4] += eps[..., 0] * mag[..., 2] + eps[..., 1] * mag[..., 1]
    bound[..., 5] += 2 * eps[..., 1] * mag[..., 2]
    for q, (i, j) in zip(range(8, 12), ((0, 6), (0, 7), (1, 6), (1, 7))):
        bound[..., q] += eps[..., i] * mag[..., j]
    win = pc > 0
    if win.any():
        vv, gg = np.nonzero(win)
        F = P.window_feature_bound(s, o, lf, (vv, gg))
        bound[vv, gg] += (pw[vv, gg] + 0.01 * pc[vv, gg])[:, None] * F
    d = np.abs(gm[..., :13] - L[..., :13])
    check = np.ones(d.shape, bool)
    check[lf["r_ambiguous"], 6:12] = False      # the reference pixel is not pinned there
    with np.errstate(divide="ignore", invalid="ignore"):
        floor = 1e-12 * big[..., None]
        rel = np.where(np.maximum(mag, floor) > 0, d / np.maximum(mag, floor), np.where(d > 0, np.inf, 0.0))
        ratio = np.where(bound > 0, d / bound, np.where(d > 0, np.inf, 0.0))
    clean = ~win[..., None] & check
    worst = np.argsort(np.where(check, ratio, 0).ravel())[::-1][:6]
    st = dict(pairs=int(win.size), window_pairs=int(win.sum()),
              window_pixel_share=float(pc.sum() / max(L[..., 13].sum(), 1)),
              r_ambiguous=int(lf["r_ambiguous"].sum()),
              rel_max_per_slot=[float(rel[..., q][clean[..., q]].max()) if clean[..., q].any() else 0.0
                                for q in range(13)],
              bound_ratio_max=float(ratio[check].max()),
              worst=[dict(v=int(k // (13 * s.n)), g=int(k // 13 % s.n), slot=int(k % 13),
                          gpu=float(gm.reshape(-1, 16)[k // 13, k % 13]), orc=float(L.reshape(-1, 15)[k // 13, k % 13]),
                          mag=float(mag.ravel()[k]), bound=float(bound.ravel()[k]),
                          npix=(float(gm.reshape(-1, 16)[k // 13, 13]), float(L.reshape(-1, 15)[k // 13, 13])),
                          pc=float(pc.ravel()[k // 13])) for k in worst])
    if tag:
        P.log_stats(tag + ":moments", st)
    assert np.all(d[check] <= bound[check]), st
    return st


def check_fitted(s, g, o, sens, tag=None, caps=None):
    """Every solved Gaussian: within the flat tolerance where the oracle pins the
    quantity to half of it, else within tol + K_SENS x the oracle's own movement;
    excluded shares within the scene's caps; statuses equal where stable."""
    caps = caps or EXCL_CAPS["default"]
    c = P.compare_outputs(s, g, o)
    st = P.summarize(c, sens)
    if tag:
        P.log_stats(tag + ":fitted", st)
    assert st["status_mismatch_stable"] == 0, st
    for k in ("pos", "scale", "angle", "cov", "covall"):
        assert st[f"{k}_fail"] == 0 and st[f"{k}_excl_fail"] == 0, (k, st)
    assert st["excluded_pos"] <= max(1, caps["pos"] * st["n_both_pos"]), st
    assert st["excluded_scale"] <= max(1, caps["scale"] * st["n_both_cov"]), st
    assert st["excluded_angle"] <= max(1, caps["angle"] * st["n_both_cov"]), st
    assert st["excluded_cov"] <= max(1, caps["cov"] * st["n_both_cov"]), st
    return st


@pytest.mark.parametrize("name", list(SCENES))
def test_moments(gpu_ready, name):
    s, g, o, _ = case(name)
    check_moments(s, o, g, tag=name)


@pytest.mark.parametrize("variant", [1, 2, 4, 5])
@pytest.mark.parametrize("name", ["tiny", "capture_sub"])
def test_raster_variants(gpu_ready, name, variant):
    """The warp-shuffle raster kernels (8x4, 8x8 and 8x16 warp blocks) and the
    persistent two-phase kernel meet the same bar as the default two-phase one.
    Their summation order and exponential differ, so pixel counts may differ only
    by blend decisions that the oracle records as lying inside the FP32 window
    (each side within that count of it)."""
    s, g2, o, sens = case(name)
    g = P.run_gpu(s, raster_variant=variant)
    check_moments(s, o, g, tag=f"{name}:variant{variant}")
    assert np.array_equal(g["pairs"], g2["pairs"])
    pc = o["moments"][..., 16]
    assert np.all(np.abs(g["view_moments"][..., 13:15].astype(np.float64)
                         - g2["view_moments"][..., 13:15]) <= 2 * pc[..., None])
    check_fitted(s, g, o, sens, tag=f"{name}:variant{variant}", caps=caps_for(s))


def check_view_solve(s, g, o, sens, tag=None):
    """Per (view, Gaussian): flags, new mean mu_2D' (Eq. 2), the affine's
    consistency A mu + b = mu_2D', and Sigma_2D' = A Sigma_2D A^T (Eq. 2).
    Records whose decision lies near a Sec. 5.1 threshold, or that hold pixels
    with a blend decision inside the FP32 window, are excluded and counted;
    records whose oracle solution moves by more than half a tolerance under
    FP32-sized perturbations are held to tol + K_SENS x that movement."""
    margin = view_margins(o)
    fo, fg = o["view_flags"], g["view_flags"]
    fstable = sens["view_flags_stable"]
    assert np.array_equal(fo[~margin & fstable], fg[~margin & fstable])
    both = (fo == 1) & (fg == 1) & ~margin & fstable
    smu, scov = sens["mu"], sens["cov2"]
    tight = both & (smu < MU_TOL_PX / 2) & (scov < COV_TOL_REL / 2)
    loose = both & ~tight
    dmu = np.linalg.norm(g["view_means"][..., :2] - o["view_mean2d"], axis=-1)
    B = g["view_B"]
    cov_g = np.stack([(B[..., 0:3] ** 2).sum(-1), (B[..., 0:3] * B[..., 4:7]).sum(-1),
                      (B[..., 4:7] ** 2).sum(-1)], -1).astype(np.float64)
    dcov = P.cov2_rel(cov_g, o["view_cov2d"])
    # [A|b] of Eq. 2 is consistent with the new mean: A mu + b = mu'
    A = g["view_affine"][..., :4].reshape(fo.shape + (2, 2)).astype(np.float64)
    b = g["view_affine"][..., 4:].astype(np.float64)
    mu_g = np.einsum("...ij,...j->...i", A, o["mean2d"]) + b
    # [A|b] is stored in FP32 in absolute pixel coordinates: A mu + b carries the
    # rounding of terms of size |A| |mu| + |b| (a few units in their last place)
    mag_ab = np.einsum("...ij,...j->...i", np.abs(A), np.abs(o["mean2d"])) + np.abs(b)
    dab = np.linalg.norm(mu_g - g["view_means"][..., :2], axis=-1) / \
        (MU_TOL_PX + 8 * 2.0 ** -24 * np.linalg.norm(mag_ab, axis=-1))
    st = dict(pairs=int(fo.size), margin=int(margin.sum()), flags_unstable=int((~fstable).sum()),
              both=int(both.sum()), sens_excluded=int(loose.sum()),
              mu_max=float(dmu[tight].max()) if tight.any() else 0.0,
              cov_max=float(dcov[tight].max()) if tight.any() else 0.0,
              ab_max=float(dab[both].max()) if both.any() else 0.0,
              mu_loose_ratio=float((dmu / (MU_TOL_PX + K * smu))[loose].max()) if loose.any() else 0.0,
              cov_loose_ratio=float((dcov / (COV_TOL_REL + K * scov))[loose].max()) if loose.any() else 0.0)
    if tag:
        P.log_stats(tag + ":view", st)
    assert st["mu_max"] < MU_TOL_PX and st["cov_max"] < COV_TOL_REL, st
    assert st["ab_max"] <= 1.0, st
    assert st["mu_loose_ratio"] <= 1.0 and st["cov_loose_ratio"] <= 1.0, st
    return st


def check_view_solve_on_gpu_moments(s, g, o, tag=None, draws=3):
    """The per-view solve (a6: Sec. 5.1 tests, Eq. 4, Eq. 2) alone, on every
    record: the GPU's own moment sums, taken back to the oracle's frame, are
    re-solved by the oracle in FP64, and the GPU's flags, mu_2D' and Sigma_2D'
    must agree.  This covers the records the end-to-end comparison leaves out
    (blend decisions inside the FP32 window change the sums themselves, not the
    solve).  Flags are compared where none of the solve's own decisions (sum w,
    det V1, lambda_min against their thresholds) lies within 5 % of its
    threshold; mu_2D' and Sigma_2D' are held to their tolerances where the FP64
    solve moves by less than half of them when the record is perturbed by a few
    FP32 roundings (2^-20 of each slot's magnitude bound: the model of
    ``parity.fp32_moment_rounding`` doubled, since the FP32 solve rounds its
    intermediate sums again), else to tol + K x that movement."""
    lf = P.library_frame(s, o)
    V, n = o["moments"].shape[:2]
    gm = g["view_moments"].astype(np.float64)[..., :15]
    Mg = P.oracle_record_from_library(gm, lf["dl"], lf["r"])
    # magnitude bounds of the GPU's own sums: the oracle's bounds (same pixels up
    # to window decisions) suffice for the rounding model
    mag = lf["mag"]
    fg = g["view_flags"]
    touched = (fg & oracle.OV_CULLED) == 0
    rng = np.random.default_rng(11)
    vv, gg = np.nonzero(touched & ~lf["r_ambiguous"])
    fo = np.zeros(len(vv), np.uint32)
    mu_o = np.zeros((len(vv), 2))
    cov_o = np.zeros((len(vv), 3))
    smu = np.zeros(len(vv))
    scov = np.zeros(len(vv))
    for j, (v, gi) in enumerate(zip(vv, gg)):
        rec = Mg[v, gi, :16]
        fl, _, m2, c2 = oracle.view_solve(rec, o["mean2d"][v, gi], o["cov2d"][v, gi])
        fo[j], mu_o[j], cov_o[j] = fl, m2, c2
        if fl != 1:
            continue
        for _ in range(draws):
            Lp = gm[v, gi].copy()
            Lp[:12] += 2.0 ** -20 * mag[v, gi, :12] * rng.uniform(-1, 1, 12)
            rp = P.oracle_record_from_library(Lp, lf["dl"][v, gi], lf["r"][v, gi])[:16]
            _, _, m3, c3 = oracle.view_solve(rp, o["mean2d"][v, gi], o["cov2d"][v, gi])
            smu[j] = max(smu[j], float(np.linalg.norm(m3 - m2)))
            scov[j] = max(scov[j], float(P.cov2_rel(c3, c2)))
    # the solve's own decisions near their thresholds (from the GPU's sums)
    R = Mg[vv, gg]
    sw = R[:, 5]
    with np.errstate(divide="ignore", invalid="ignore"):
        mx, my = R[:, 2] / sw, R[:, 4] / sw
        cxx, cxy, cyy = R[:, 0] / sw - mx * mx, R[:, 1] / sw - mx * my, R[:, 3] / sw - my * my
        tr, dt = cxx + cyy, cxx * cyy - cxy * cxy
        lmin = 0.5 * (tr - np.sqrt(np.maximum(tr * tr - 4 * dt, 0)))
        det = sw ** 3 * dt
    near_thr = near(sw, 1e-3) | near(det, 1e-12) | near(lmin, 1e-4)
    fgj = fg[vv, gg]
    cmp = ~near_thr
    both = cmp & (fo == 1) & (fgj == 1)
    dmu = np.linalg.norm(g["view_means"][vv, gg, :2] - mu_o, axis=-1)
    B = g["view_B"][vv, gg]
    cov_g = np.stack([(B[:, 0:3] ** 2).sum(-1), (B[:, 0:3] * B[:, 4:7]).sum(-1), (B[:, 4:7] ** 2).sum(-1)], -1)
    dcov = P.cov2_rel(cov_g.astype(np.float64), cov_o)
    tight = both & (smu < MU_TOL_PX / 2) & (scov < COV_TOL_REL / 2)
    loose = both & ~tight
    st = dict(records=int(len(vv)), near_threshold=int(near_thr.sum()),
              flag_mismatch=int((fo[cmp] != fgj[cmp]).sum()), both=int(both.sum()), sens_excluded=int(loose.sum()),
              mu_max=float(dmu[tight].max()) if tight.any() else 0.0,
              cov_max=float(dcov[tight].max()) if tight.any() else 0.0,
              mu_loose_ratio=float((dmu / (MU_TOL_PX + K * smu))[loose].max()) if loose.any() else 0.0,
              cov_loose_ratio=float((dcov / (COV_TOL_REL + K * scov))[loose].max()) if loose.any() else 0.0)
    if tag:
        P.log_stats(tag + ":a6_on_gpu_moments", st)
    assert st["flag_mismatch"] == 0, st
    assert st["mu_max"] < MU_TOL_PX and st["cov_max"] < COV_TOL_REL, st
    assert st["mu_loose_ratio"] <= 1.0 and st["cov_loose_ratio"] <= 1.0, st
    return st


K = P.K_SENS


@pytest.mark.parametrize("name", list(SCENES))
def test_view_solve(gpu_ready, name):
    s, g, o, sens = case(name)
    st = check_view_solve(s, g, o, sens, tag=name)
    assert st["margin"] <= VIEW_MARGIN_CAP * st["pairs"], st


@pytest.mark.parametrize("name", list(SCENES))
def test_view_solve_on_gpu_moments(gpu_ready, name):
    s, g, o, _ = case(name)
    check_view_solve_on_gpu_moments(s, g, o, tag=name)


@pytest.mark.parametrize("name", list(SCENES))
def test_fitted_gaussians(gpu_ready, name):
    s, g, o, sens = case(name)
    check_fitted(s, g, o, sens, tag=name, caps=caps_for(s))


@pytest.mark.parametrize("name", ["tiny", "capture_sub"])
def test_render(gpu_ready, name):
    import torch
    import paper_2604_02586_b300 as tsp
    s = SCENES[name]()
    d = P.to_device(s)
    with tsp.Context(0) as ctx:
        rgb, T = ctx.render(d["means_opacity"], d["quats"], d["scales"],
                            torch.from_numpy(s.sh).cuda(), s.sh_degree, s, sync=True)
    orgb, oT, fl = oracle.render(s)
    for v in range(s.num_views):
        m = fl[v] == 0
        assert (~m).mean() <= RENDER_WINDOW_CAP
        ec = np.abs(rgb[v].cpu().numpy() - orgb[v]).max(-1)[m]
        eT = np.abs(T[v].cpu().numpy() - oT[v])[m]
        assert ec.max() < PIX_TOL and eT.max() < PIX_TOL, (ec.max(), eT.max())


def test_integer_outputs_are_deterministic(gpu_ready):
    s = SCENES["tiny"]()
    a, b = P.run_gpu(s), P.run_gpu(s)
    for k in ("rect", "depth", "touched", "tile_off", "pairs", "view_flags"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["view_moments"][..., 13], b["view_moments"][..., 13])
    np.testing.assert_allclose(a["means"], b["means"], rtol=0, atol=1e-5)


def test_host_entry_point_matches_device(gpu_ready):
    import paper_2604_02586_b300 as tsp
    s, g, _, _ = case("tiny")
    with tsp.Context(0) as ctx:
        h = ctx.fit_motion_host(s.means_opacity, s.quats, s.scales, s, s.disp, s.vis)
    assert np.array_equal(h["status"] & 0xFF, g["status"] & 0xFF)
    np.testing.assert_allclose(h["means"], g["means"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(h["scales"], g["scales"], rtol=1e-4, atol=0)


@pytest.mark.parametrize("n,views", [(1, 3), (2, 3), (301, 4), (300, 0), (0, 3)])
def test_host_entry_point_edges(gpu_ready, n, views):
    """The host-buffer call streams its results back in two halves of the
    Gaussians (the first half may be empty); without views it copies them back
    whole.  Both agree with the device call."""
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 5, n=max(n, 1), views=max(views, 1))
    if n == 0:
        s = synth.make_scene("tiny", 5, n=0, views=views)
    if views == 0:
        s = s.subset_views([])
    with tsp.Context(0) as ctx:
        g = P.run_gpu(s, ctx=ctx, inspect=False)
        h = ctx.fit_motion_host(s.means_opacity, s.quats, s.scales, s, s.disp, s.vis)
    assert h["means"].shape == (n, 4) and h["status"].shape == (n,)
    assert np.array_equal(h["status"] & 0xFF, g["status"] & 0xFF)
    np.testing.assert_allclose(h["means"], g["means"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(h["scales"], g["scales"], rtol=1e-4, atol=0)
    if views == 0:
        assert np.array_equal(h["means"], s.means_opacity)


def test_empty_and_degenerate_inputs(gpu_ready):
    import torch
    import paper_2604_02586_b300 as tsp
    base = synth.make_scene("tiny", 2, n=300, views=3)
    with tsp.Context(0) as ctx:
        # no Gaussians
        e = synth.make_scene("tiny", 2, n=0, views=3)
        r = P.run_gpu(e, ctx=ctx, inspect=False)
        assert r["means"].shape == (0, 4)
        # no views: every Gaussian keeps its input, FEW_VIEWS
        r = P.run_gpu(base.subset_views([]), ctx=ctx, inspect=False)
        assert np.all(r["status"] & tsp.TSP.FEW_VIEWS)
        assert np.array_equal(r["means"], base.means_opacity)
        assert np.array_equal(r["quats"], base.quats)
        # everything behind the cameras: all culled
        far = synth.make_scene("tiny", 2, n=300, views=3)
        far.means_opacity[:, :3] += 100.0
        r = P.run_gpu(far, ctx=ctx, inspect=True)
        assert int(r["counts"][0]) == 0 and np.all(r["touched"] == 0)
        assert np.all(r["view_flags"] & tsp.TSP.VIEW_CULLED)
        assert np.array_equal(r["means"], far.means_opacity)
        # no valid track anywhere: nothing accumulates
        dark = synth.make_scene("tiny", 2, n=300, views=3)
        for v in dark.vis:
            v[:] = 0
        r = P.run_gpu(dark, ctx=ctx, inspect=False)
        assert np.all(r["view_moments"][..., 0] == 0) and np.all(r["status"] & tsp.TSP.FEW_VIEWS)


def test_many_views_and_ragged_tiles(gpu_ready):
    s = synth.make_scene("tiny", 12, n=600, views=32, width=72, height=40, focal=60.0)
    g = P.run_gpu(s)
    o = oracle.fit_motion(s)
    off, ent = oracle.bin_lists(s)
    assert np.array_equal(g["pairs"], ent)
    check_moments(s, o, g, tag="many_views")
    check_fitted(s, g, o, P.sensitivity(s, o), tag="many_views")


def test_pair_overflow_is_reported_then_recovered(gpu_ready):
    import paper_2604_02586_b300 as tsp
    s, g, _, _ = case("capture_sub")          # K = 4.3e5 pairs > the 65,536 minimum
    d = P.to_device(s)
    with tsp.Context(0, async_pairs=1, pair_capacity=1000) as ctx:
        ctx.fit_motion(d["means_opacity"], d["quats"], d["scales"], s, d["disp"], d["vis"])
        with pytest.raises(tsp.TspError) as ei:
            ctx.sync()
        assert ei.value.status == tsp.TSP.ERR_OVERFLOW
        out = ctx.fit_motion(d["means_opacity"], d["quats"], d["scales"], s, d["disp"], d["vis"],
                             sync=True)
        assert int(ctx.inspect(tsp.TSP.I_COUNTS)[3]) == 0
    assert np.array_equal(out["status"].cpu().numpy().view(np.uint32) & 0xFF, g["status"] & 0xFF)


def test_bad_pointers_are_rejected_before_launch(gpu_ready):
    import torch
    import paper_2604_02586_b300 as tsp
    s = SCENES["tiny"]()
    d = P.to_device(s)
    L = tsp.lib()
    with tsp.Context(0) as ctx:
        n = s.n
        flat = torch.zeros(4 * n + 1, device="cuda")
        mis = flat[1:]                                    # 4-byte aligned only
        host = np.zeros((n, 4), np.float32)
        carr, V = tsp.cameras_from(s.width, s.height, s.fx, s.fy, s.cx, s.cy, s.R, s.t)
        tr = (tsp.ViewTracks * V)()
        for v in range(V):
            tr[v].disp, tr[v].vis = d["disp"][v].data_ptr(), d["vis"][v].data_ptr()
        outs = [torch.empty((n, 4), device="cuda") for _ in range(3)] + [torch.empty(n, dtype=torch.int32, device="cuda")]
        r = tsp.Result(*[o.data_ptr() for o in outs], None, None, None)
        for bad in (mis.data_ptr(), host.ctypes.data):
            g = tsp.Gaussians(n, bad, d["quats"].data_ptr(), d["scales"].data_ptr())
            st = L.tsp_fit_motion(ctx._h, C.byref(g), carr, V, tr, C.byref(r), None)
            assert st == tsp.TSP.ERR_INVALID_ARG
        g = tsp.Gaussians(n, d["means_opacity"].data_ptr(), d["quats"].data_ptr(), d["scales"].data_ptr())
        assert L.tsp_fit_motion(ctx._h, C.byref(g), carr, 33, tr, C.byref(r), None) == tsp.TSP.ERR_INVALID_ARG


def test_sync_timeout_is_reported_and_the_context_recovers(gpu_ready):
    """tsp_sync with a time limit returns TIMEOUT while the stream is still
    busy (here with a bounded spin of about 0.1 s queued before the fit), leaves
    the work running, and a later full sync and the next call succeed."""
    import torch
    import paper_2604_02586_b300 as tsp
    s, g, _, _ = case("tiny")
    d = P.to_device(s)
    # async_pairs: the call only enqueues (no host wait for the pair count)
    with tsp.Context(0, async_pairs=1, pair_capacity=1 << 20) as ctx:
        torch.cuda._sleep(200_000_000)              # ~0.1 s of GPU cycles, then it ends
        out = ctx.fit_motion(d["means_opacity"], d["quats"], d["scales"], s, d["disp"], d["vis"])
        with pytest.raises(tsp.TspError) as e:
            ctx.sync(timeout_ms=1)
        assert e.value.status == tsp.TSP.ERR_TIMEOUT
        ctx.sync()
        st = out["status"].cpu().numpy().view(np.uint32)
        assert np.array_equal(st & 0xFF, g["status"] & 0xFF)
        r = P.run_gpu(s, ctx=ctx, inspect=False)
        assert np.array_equal(r["status"] & 0xFF, g["status"] & 0xFF)


def test_options_are_validated(gpu_ready):
    import paper_2604_02586_b300 as tsp
    for bad in ({"cov_rcond_min": 0.0}, {"cov_rcond_min": 1.0}, {"raster_variant": 3},
                {"tile_w": 32}, {"tile_w": 8, "tile_h": 32}, {"tile_w": 32, "tile_h": 8, "raster_variant": 2},
                {"det_min": -1.0}, {"min_views": -1}):
        with pytest.raises(tsp.TspError):
            tsp.Context(0, **bad)
    for ok in ({"cov_rcond_min": 1e-12}, {"raster_variant": 4}, {"tile_w": 32, "tile_h": 8},
               {"tile_w": 32, "tile_h": 8, "raster_variant": 5}):
        tsp.Context(0, **ok).close()


@pytest.mark.parametrize("name", ["tiny", "capture_sub"])
def test_wide_tiles_bin_and_fit(gpu_ready, name):
    """32 x 8 tiles (four 8x8 warp blocks in a row), with both two-phase raster
    kernels: keys and tile lists equal the oracle's for that tile shape bit for
    bit, and moments and fitted Gaussians meet the 16 x 16 bar."""
    s = SCENES[name]()
    opt = oracle.default_options(tile=(32, 8))
    o = oracle.fit_motion(s, opt)
    sens = P.sensitivity(s, o, options=opt)
    k = oracle.keys(s, tile=(32, 8))
    off, ent = oracle.bin_lists(s, tile=(32, 8))
    for variant in (0, 5):
        g = P.run_gpu(s, tile_w=32, tile_h=8, raster_variant=variant)
        assert np.array_equal(g["rect"].astype(np.int32), k["rect"])
        assert np.array_equal(g["touched"], k["tiles_touched"])
        assert int(g["counts"][0]) == len(ent) and int(g["counts"][3]) == 0
        assert np.array_equal(g["tile_off"].astype(np.int64), off)
        assert np.array_equal(g["pairs"], ent)
        check_moments(s, o, g, tag=f"{name}:32x8:variant{variant}", tile=(32, 8))
        check_fitted(s, g, o, sens, tag=f"{name}:32x8:variant{variant}", caps=caps_for(s))


@pytest.mark.parametrize("ragged", [False, True])
def test_wide_tiles_render(gpu_ready, ragged):
    """The colour render with 32 x 8 tiles against the oracle's; the ragged case
    (100 x 70 pixels) leaves partial tiles in both directions."""
    import torch
    import paper_2604_02586_b300 as tsp
    s = (synth.make_scene("tiny", 13, n=700, views=3, width=100, height=70, focal=80.0) if ragged
         else SCENES["capture_sub"]())
    d = P.to_device(s)
    with tsp.Context(0, tile_w=32, tile_h=8) as ctx:
        rgb, T = ctx.render(d["means_opacity"], d["quats"], d["scales"],
                            torch.from_numpy(s.sh).cuda(), s.sh_degree, s, sync=True)
    orgb, oT, fl = oracle.render(s, tile=(32, 8))
    for v in range(s.num_views):
        m = fl[v] == 0
        assert (~m).mean() <= RENDER_WINDOW_CAP
        ec = np.abs(rgb[v].cpu().numpy() - orgb[v]).max(-1)[m]
        eT = np.abs(T[v].cpu().numpy() - oT[v])[m]
        assert ec.max() < PIX_TOL and eT.max() < PIX_TOL, (ec.max(), eT.max())


def test_full_capture_sampled(gpu_ready):
    """The bench's workload and launch configuration: 200k Gaussians x 18 views at
    1352x1014, pair buffer sized once and calls asynchronous; 200 sampled
    Gaussians recomputed by the oracle."""
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("capture", 2)
    d = P.to_device(s)
    with tsp.Context(0) as probe:
        probe.fit_motion(d["means_opacity"], d["quats"], d["scales"], s, d["disp"], d["vis"], sync=True)
        K = int(probe.inspect(tsp.TSP.I_COUNTS)[0])
    with tsp.Context(0, async_pairs=1, pair_capacity=int(K * 1.1) + 1024) as ctx:
        g = P.run_gpu(s, ctx=ctx, inspect=True)
    assert int(g["counts"][3]) == 0
    ids = np.sort(np.random.default_rng(0).choice(s.n, 200, replace=False))
    o = oracle.fit_motion(s, sample=ids, per_view=True)
    sens = P.sensitivity(s, o, sample=ids)
    st = P.summarize(P.compare_outputs(s, g, o, ids=ids), sens)
    P.log_stats("full_capture_sampled", st)
    caps = EXCL_CAPS["full_capture"]
    assert st["status_mismatch_stable"] == 0, st
    for k in ("pos", "scale", "angle", "cov", "covall"):
        assert st[f"{k}_fail"] == 0 and st[f"{k}_excl_fail"] == 0, (k, st)
    assert st["excluded_pos"] <= max(1, caps["pos"] * st["n_both_pos"]), st
    assert st["excluded_scale"] <= max(1, caps["scale"] * st["n_both_cov"]), st
    assert st["excluded_angle"] <= max(1, caps["angle"] * st["n_both_cov"]), st
    assert st["excluded_cov"] <= max(1, caps["cov"] * st["n_both_cov"]), st
