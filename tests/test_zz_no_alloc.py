"""tsp_sort_tiles_noalloc: the per-tile depth sort for callers that cannot
allocate device memory (a memory-capped tenant of a shared GPU, a host whose own
allocator owns the device memory, a loop that cannot afford an allocation's
device-wide synchronization).

The entry point is called through the C ABI on shuffled copies of the tile lists
that tsp_fit_motion produced, twice in a row, and must give back exactly the
lists tsp_fit_motion sorted (integer keys: bit-exact).  A dense scene makes some
lists longer than 4096 keys, so the merge through the library's static scratch
array runs.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import synth
from tests import parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu_ready():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02586_b300 import build as tbuild
    tbuild.build()
    return True


def reference_lists(scene):
    g = P.run_gpu(scene)
    return g["tile_off"], g["pairs"]


def shuffled(off, keys, seed):
    rng = np.random.default_rng(seed)
    out = keys.copy()
    for t in range(len(off) - 1):
        b, e = int(off[t]), int(off[t + 1])
        if e - b > 1:
            out[b:e] = out[b:e][rng.permutation(e - b)]
    return out


def sort_noalloc(off, keys):
    import ctypes as C
    import torch
    import paper_2604_02586_b300 as tsp
    dk = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    do = torch.from_numpy(off.astype(np.int32)).cuda()
    st = tsp.lib().tsp_sort_tiles_noalloc(C.c_void_p(dk.data_ptr()), C.c_void_p(do.data_ptr()),
                                          len(off) - 1, len(keys), None)
    assert st == tsp.TSP.OK
    torch.cuda.synchronize()
    return dk.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("dense", [False, True])
def test_noalloc_sort_matches_fit_motion_lists(gpu_ready, dense):
    s = synth.make_scene("tiny", 3, n=30000 if dense else 2000, views=2 if dense else 4)
    if dense:
        s.means_opacity[:, :3] *= 0.05          # one-tile clusters: lists of ~30,000 keys
    off, ref = reference_lists(s)
    if dense:
        assert np.diff(off).max() > 4096
    for seed in (1, 2):                         # two calls in a row share the scratch
        got = sort_noalloc(off, shuffled(off, ref, seed))
        assert np.array_equal(got, ref)


def test_noalloc_sort_repeated_keys_across_runs(gpu_ready):
    """Equal keys in both runs of a merge (lists longer than 4096 keys drawn from
    a few hundred values, so every run boundary splits groups of equal keys):
    the result is the ascending order of the input, nothing lost or duplicated."""
    rng = np.random.default_rng(5)
    sizes = [9000, 1, 0, 4097, 300, 16384 + 17]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    keys = np.concatenate([(rng.integers(0, 257, m).astype(np.uint64) << np.uint64(32)) |
                           rng.integers(0, 3, m).astype(np.uint64) for m in sizes])
    want = keys.copy()
    for t in range(len(sizes)):
        want[off[t]:off[t + 1]].sort()
    for _ in range(2):
        got = sort_noalloc(off, keys)
        assert np.array_equal(got, want)


def test_noalloc_sort_rejects_oversized_input(gpu_ready):
    import paper_2604_02586_b300 as tsp
    too_many = (1 << 20) + 1
    st = tsp.lib().tsp_sort_tiles_noalloc(None, None, 1, too_many, None)
    assert st == tsp.TSP.ERR_INVALID_ARG
