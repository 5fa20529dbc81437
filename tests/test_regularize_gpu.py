"""Motion regularization (Sec. 4.5) on a B300 through the C ABI, against the
oracle: nearest neighbours bit-exact (FP32 distance, ties by index) on random,
clustered, lattice (many exact ties), flat and duplicated point sets with dense,
sparse, empty and single-member masks; static flags exact; regularized means
within 1e-4 of the scene extent, scales within 1e-4 relative and rotations within
1e-3 rad of the oracle's.

Rotation changes enter the filter as Euler angles.  Where an angle lies next to
the +-pi branch cut or the pitch next to +-pi/2 (gimbal lock), FP32 and FP64 may
take the conversion to different, equally valid branches and the median then
picks different values; rotations are compared where every angle in the
Gaussian's filter window is 1e-3 away from those places (all of them for the
inputs of ``motion_pair``, which turn by at most 0.2 rad).
"""
import zlib

import numpy as np
import pytest

import oracle
import synth
from tests import parity as P
from tests.parity import rot_angle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02586_b300 import build as tbuild
    tbuild.build()
    import paper_2604_02586_b300 as tsp
    c = tsp.Context(0)
    yield c
    c.close()


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def points(kind, n, rng):
    return synth.point_set(kind, n, rng)


def mask_of(kind, n, rng):
    if kind == "all":
        return np.ones(n, np.uint8)
    if kind == "half":
        return (rng.random(n) < 0.5).astype(np.uint8)
    if kind == "sparse":
        m = (rng.random(n) < 0.01).astype(np.uint8)
        m[rng.integers(0, n)] = 1
        return m
    if kind == "none":
        return np.zeros(n, np.uint8)
    if kind == "one":
        m = np.zeros(n, np.uint8)
        m[n // 3] = 1
        return m
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "clustered", "lattice", "flat", "duplicates", "offset", "spheres_far",
                                  "blobs"])
@pytest.mark.parametrize("mkind", ["all", "half", "sparse", "none", "one"])
def test_knn_bit_exact(ctx, kind, mkind):
    rng = np.random.default_rng(zlib.crc32(f"{kind}/{mkind}".encode()))
    n = 3001
    mo = points(kind, n, rng)
    mask = mask_of(mkind, n, rng)
    for k in (1, 8, 16):
        got = ctx.knn(cuda(mo), cuda(mask), k, sync=True).cpu().numpy()
        want = oracle.knn(mo, mask, k)
        bad = np.nonzero((got != want).any(1))[0]
        assert bad.size == 0, (k, bad[:5], got[bad[:2]], want[bad[:2]])


@pytest.mark.parametrize("n", [0, 1, 2, 9])
def test_knn_tiny(ctx, n):
    rng = np.random.default_rng(n)
    mo = points("uniform", max(n, 1), rng)[:n]
    mask = np.ones(n, np.uint8)
    got = ctx.knn(cuda(mo), cuda(mask), 8, sync=True).cpu().numpy()
    assert got.shape == (n, 8)
    np.testing.assert_array_equal(got, oracle.knn(mo, mask, 8))


def test_knn_path_follows_the_point_distribution(ctx):
    """A near-uniform set is searched on the grid; sets whose density varies by
    orders of magnitude switch to the BVH (both give the exact lists)."""
    import paper_2604_02586_b300 as tsp
    rng = np.random.default_rng(5)
    n = 20000
    for kind, want in (("uniform", 0), ("lattice", 0), ("blobs", 1), ("spheres_far", 1)):
        mo = points(kind, n, rng)
        mask = np.ones(n, np.uint8)
        got = ctx.knn(cuda(mo), cuda(mask), 8, sync=True).cpu().numpy()
        assert ctx.inspect(tsp.TSP.I_KNN_PATH)[0] == want, kind
        q = rng.choice(n, 200, replace=False)
        X = mo[:, :3]
        for i in q:
            d = X[i] - X
            d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
            d2[i] = np.inf
            np.testing.assert_array_equal(got[i], np.lexsort((np.arange(n), d2))[:8])


@pytest.mark.parametrize("kind", ["uniform", "spheres_far"])
def test_knn_large_sampled(ctx, kind):
    """200,000 points, uniform in a 4-unit box (the capture workload's Gaussians)
    or on sphere surfaces with a far field: sampled queries against an FP32 brute
    force over all points."""
    rng = np.random.default_rng(77)
    n, k = 200_000, 8
    mo = points(kind, n, rng)
    mask = (rng.random(n) < 0.85).astype(np.uint8)
    got = ctx.knn(cuda(mo), cuda(mask), k, sync=True).cpu().numpy()
    q = rng.choice(n, 300, replace=False)
    X = mo[:, :3]
    for i in q:
        d = X[i] - X                                                  # FP32, as the pinned distance
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        d2[mask == 0] = np.inf
        d2[i] = np.inf
        order = np.lexsort((np.arange(n), d2))[:k]
        np.testing.assert_array_equal(got[i], order)


def euler_window_ok(before, after, nbr_lists, has, tol=1e-3):
    """Gaussians whose own and neighbours' rotation-change Euler angles are all
    away from the branch cuts (FP64)."""
    def rot(q):
        q = q.astype(np.float64) / np.linalg.norm(q, axis=1, keepdims=True)
        w, x, y, z = q.T
        return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                         np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                         np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    D = rot(after[1]) @ np.transpose(rot(before[1]), (0, 2, 1))
    ex = np.arctan2(D[:, 2, 1], D[:, 2, 2])
    ey = np.arcsin(np.clip(-D[:, 2, 0], -1, 1))
    ez = np.arctan2(D[:, 1, 0], D[:, 0, 0])
    safe = (np.pi - np.abs(ex) > tol) & (np.pi - np.abs(ez) > tol) & (np.pi / 2 - np.abs(ey) > tol)
    ok = safe.copy()
    for j in range(nbr_lists.shape[1]):
        nb = nbr_lists[:, j]
        ok &= np.where(nb >= 0, safe[np.maximum(nb, 0)], True)
    return ok


def compare_regularized(got, want, before, extent, rot_ok):
    np.testing.assert_array_equal(got["flags"], want["flags"])
    dpos = np.abs(got["means_opacity"][:, :3].astype(np.float64) - want["means_opacity"][:, :3]).max(1)
    assert dpos.max() <= 1e-4 * extent, dpos.max()
    np.testing.assert_array_equal(got["means_opacity"][:, 3], before[0][:, 3])
    srel = (np.abs(got["scales"][:, :3].astype(np.float64) - want["scales"][:, :3]) /
            np.maximum(np.abs(want["scales"][:, :3]), 1e-6)).max(1)
    assert srel.max() <= 1e-4, srel.max()
    qa = got["quats"].astype(np.float64)
    ang = rot_angle(qa, want["quats"])
    assert ang[rot_ok].max(initial=0) <= 1e-3, ang[rot_ok].max()
    assert np.abs(np.linalg.norm(qa, axis=1) - 1).max() < 1e-5
    # the sign stays on the side of the input quaternion
    assert ((qa * before[1]).sum(1) >= 0).all()


def run_reg(ctx, inp, k=8, V=None):
    import torch
    before = tuple(cuda(a) for a in inp["before"])
    n = inp["before"][0].shape[0]
    V = inp["npix"].shape[0] if V is None else V
    mom = np.zeros((V, n, 16), np.float32)
    mom[:, :, 13] = inp["npix"][:V]
    mom[:, :, 14] = inp["nstat"][:V]
    fitted = dict(means=cuda(inp["after"][0]), quats=cuda(inp["after"][1]), scales=cuda(inp["after"][2]),
                  status=cuda(inp["status"].view(np.int32)))
    out = ctx.regularize(before, fitted, V, view_moments=cuda(mom), k=k, neighbours=True, sync=True)
    torch.cuda.synchronize()
    res = {key: v.cpu().numpy() for key, v in out.items()}
    res["flags"] = res["flags"].view(np.uint32)
    return res


@pytest.mark.parametrize("seed,n,k,lattice", [(1, 5000, 8, False), (2, 5000, 8, True), (3, 3000, 16, False),
                                               (4, 2000, 1, False), (5, 4097, 5, True)])
def test_regularize_matches_oracle(ctx, seed, n, k, lattice):
    inp = synth.motion_pair(n, views=4, seed=seed, lattice=lattice)
    got = run_reg(ctx, inp, k)
    is_static = oracle.static_flags(inp["npix"], inp["nstat"])
    np.testing.assert_array_equal(got["flags"] & 1, is_static)
    has_pos = ((inp["status"] & 1) > 0) & (is_static == 0)
    has_cov = ((inp["status"] & 2) > 0) & (is_static == 0)
    mo0 = inp["before"][0]
    np.testing.assert_array_equal(got["nbr_pos"], oracle.knn(mo0, has_pos.astype(np.uint8), k))
    np.testing.assert_array_equal(got["nbr_cov"], oracle.knn(mo0, has_cov.astype(np.uint8), k))
    want = oracle.regularize(inp["before"], inp["after"], inp["status"], is_static, k)
    rot_ok = euler_window_ok(inp["before"], inp["after"], got["nbr_cov"], has_cov)
    assert rot_ok.mean() > 0.99
    compare_regularized(got, want, inp["before"], 4.0, rot_ok)
    # every case of the rule occurs
    for bit in (1, 2, 4, 8, 16):
        assert (got["flags"] & bit).any(), bit


def test_regularize_edge_cases(ctx):
    import paper_2604_02586_b300 as tsp
    inp = synth.motion_pair(600, views=3, seed=9)
    n = 600
    # every Gaussian static: outputs are the inputs (quaternions normalised)
    inp_s = dict(inp, npix=np.full((3, n), 20, np.float32), nstat=np.full((3, n), 20, np.float32))
    got = run_reg(ctx, inp_s)
    assert (got["flags"] == tsp.TSP.REG_STATIC).all()
    np.testing.assert_array_equal(got["means_opacity"], inp["before"][0])
    np.testing.assert_allclose(got["scales"], inp["before"][2], rtol=0, atol=0)
    # nothing solved: nobody moves, nothing is flagged but the static ones
    inp_0 = dict(inp, status=np.zeros(n, np.uint32))
    got = run_reg(ctx, inp_0)
    assert ((got["flags"] & ~np.uint32(1)) == 0).all()
    np.testing.assert_array_equal(got["means_opacity"], inp["before"][0])
    assert (got["nbr_pos"] == -1).all() and (got["nbr_cov"] == -1).all()
    # no views: no static Gaussians
    got = run_reg(ctx, inp, V=0)
    assert ((got["flags"] & 1) == 0).all()
    want = oracle.regularize(inp["before"], inp["after"], inp["status"], np.zeros(n, np.uint8), 8)
    np.testing.assert_array_equal(got["flags"], want["flags"])
    # k larger than the number of members: -1 padding
    inp_1 = dict(inp, status=np.zeros(n, np.uint32))
    inp_1["status"][:3] = 3
    got = run_reg(ctx, inp_1, k=16)
    assert ((got["nbr_pos"] >= 0).sum(1) <= 3).all()
    is_static = oracle.static_flags(inp_1["npix"], inp_1["nstat"])
    want = oracle.regularize(inp_1["before"], inp_1["after"], inp_1["status"], is_static, 16)
    np.testing.assert_array_equal(got["flags"], want["flags"])
    np.testing.assert_allclose(got["means_opacity"], want["means_opacity"], rtol=0, atol=4e-4)


def oracle_fit_inputs(s):
    """The oracle's own fit of scene s as regularization inputs: fitted Gaussians
    (float32 [n, 4]), status and per-view moments in the library layout."""
    o = oracle.fit_motion(s, per_view=True)
    n = s.n
    mo = np.zeros((n, 4), np.float32)
    mo[:, :3] = o["out_mean"]
    mo[:, 3] = s.means_opacity[:, 3]
    sc = np.zeros((n, 4), np.float32)
    sc[:, :3] = o["out_scale"]
    after = (mo, o["out_quat"].astype(np.float32), sc)
    mom = np.zeros(o["moments"].shape[:2] + (16,), np.float32)
    mom[..., :15] = P.library_frame(s, o)["mom"]
    return after, o["out_status"].astype(np.uint32), mom


def test_regularize_after_a_fit_uses_the_context_moments(ctx):
    """The whole chain on a fitted frame: fit_motion, then regularize with the
    moments the context kept (view_moments=None) equals regularize with the
    moments the fit returned; a frame whose neighbours' fit is wrong is not
    needed for this check (GPU against GPU)."""
    import torch
    import paper_2604_02586_b300 as tsp
    s = synth.make_scene("tiny", 8, n=3000)
    from tests.parity import to_device
    d = to_device(s)
    out = ctx.fit_motion(d["means_opacity"], d["quats"], d["scales"], s, d["disp"], d["vis"], view_moments=True)
    ctx.sync()
    before = (d["means_opacity"], d["quats"], d["scales"])
    r1 = ctx.regularize(before, out, s.num_views, neighbours=True, sync=True)
    r2 = ctx.regularize(before, out, s.num_views, view_moments=out["view_moments"], neighbours=True, sync=True)
    torch.cuda.synchronize()
    for key in r1:
        np.testing.assert_array_equal(r1[key].cpu().numpy(), r2[key].cpu().numpy())
    fl = r1["flags"].cpu().numpy().view(np.uint32)
    assert (fl & (tsp.TSP.REG_POS_MEDIAN | tsp.TSP.REG_POS_PROPAGATED)).any()
    # another n than the last fit's: the context's moments do not apply
    with pytest.raises(tsp.TspError):
        ctx.regularize(tuple(t[:100] for t in before), {key: out[key][:100] for key in out}, s.num_views)


def test_regularize_on_the_oracle_fit_matches_the_oracle(ctx):
    """Regularization of a fitted frame (the oracle's fit: realistic status bits,
    static counters and motions) on the GPU and in the oracle, from the same
    inputs, none of which comes from the CUDA path."""
    s = synth.make_scene("tiny", 8, n=3000)
    after, status, mom = oracle_fit_inputs(s)
    before = (s.means_opacity, s.quats, s.scales)
    fitted = dict(means=cuda(after[0]), quats=cuda(after[1]), scales=cuda(after[2]),
                  status=cuda(status.view(np.int32)))
    r = ctx.regularize(tuple(cuda(a) for a in before), fitted, s.num_views, view_moments=cuda(mom),
                       neighbours=True, sync=True)
    got = {key: v.cpu().numpy() for key, v in r.items()}
    got["flags"] = got["flags"].view(np.uint32)
    is_static = oracle.static_flags(mom[:, :, 13], mom[:, :, 14])
    want = oracle.regularize(before, after, status, is_static, 8)
    has_pos = ((status & 1) > 0) & (is_static == 0)
    has_cov = ((status & 2) > 0) & (is_static == 0)
    np.testing.assert_array_equal(got["nbr_pos"], oracle.knn(s.means_opacity, has_pos.astype(np.uint8), 8))
    np.testing.assert_array_equal(got["nbr_cov"], oracle.knn(s.means_opacity, has_cov.astype(np.uint8), 8))
    rot_ok = euler_window_ok(before, after, got["nbr_cov"], has_cov)
    compare_regularized(got, want, before, s.extent, rot_ok)
    assert (got["flags"] & 6).any()


def test_regularize_rejects_bad_arguments(ctx):
    import paper_2604_02586_b300 as tsp
    inp = synth.motion_pair(100, views=2, seed=3)
    before = tuple(cuda(a) for a in inp["before"])
    fitted = dict(means=cuda(inp["after"][0]), quats=cuda(inp["after"][1]), scales=cuda(inp["after"][2]),
                  status=cuda(inp["status"].view(np.int32)))
    mom = cuda(np.zeros((2, 100, 16), np.float32))
    for bad in (dict(k=0), dict(k=17), dict(static_frac=1.5), dict(static_min_views=0)):
        with pytest.raises(tsp.TspError):
            ctx.regularize(before, fitted, 2, view_moments=mom, **bad)
    with pytest.raises(tsp.TspError):
        ctx.knn(before[0], cuda(np.ones(100, np.uint8)), 0)


def test_regularize_replays_in_a_cuda_graph(ctx):
    """No host wait inside: the call captures into a CUDA graph, and replays on
    new inputs give the direct call's results."""
    import torch
    inp = synth.motion_pair(4000, views=4, seed=12)
    ref = run_reg(ctx, inp)
    n = 4000
    before = tuple(cuda(a) for a in inp["before"])
    fitted = dict(means=cuda(inp["after"][0]), quats=cuda(inp["after"][1]), scales=cuda(inp["after"][2]),
                  status=cuda(inp["status"].view(np.int32)))
    mom = np.zeros((4, n, 16), np.float32)
    mom[:, :, 13], mom[:, :, 14] = inp["npix"], inp["nstat"]
    mom = cuda(mom)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        ctx.regularize(before, fitted, 4, view_moments=mom)                # workspace exists before capture
    torch.cuda.current_stream().wait_stream(st)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out = ctx.regularize(before, fitted, 4, view_moments=mom)
    for key in ("means", "quats", "scales"):
        fitted[key].zero_()
    g.replay()
    torch.cuda.synchronize()
    z = out["means_opacity"].cpu().numpy()
    assert not np.array_equal(z, ref["means_opacity"])                    # zeroed inputs moved things
    fitted["means"].copy_(cuda(inp["after"][0]))
    fitted["quats"].copy_(cuda(inp["after"][1]))
    fitted["scales"].copy_(cuda(inp["after"][2]))
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["means_opacity"].cpu().numpy(), ref["means_opacity"])
    np.testing.assert_array_equal(out["flags"].cpu().numpy().view(np.uint32), ref["flags"])
