"""The scratch-free bin/sort entry point against the workspace one.

gsparc_bin_sort_noalloc serves callers that cannot call cudaMalloc (a
real-time loop that must not take an allocation's device-wide
synchronisation after start-up, or a plugin handed buffers but no
allocator).  Its scratch is one fixed device array inside the library, so
two calls in a row must each give exactly what gsparc_bin_sort gives with a
caller workspace: the second call must not see the first call's leftovers.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceScene, Renderer


def test_noalloc_rejects_sizes_above_its_limit_on_the_host():
    L = G.lib()
    v = G.make_view(90, 360)
    vp = ctypes.c_void_p
    rc = L.gsparc_bin_sort_noalloc(ctypes.byref(v), G.GSPARC_NOALLOC_MAX_N + 1, vp(256), 1024, vp(256),
                                   None, vp(256), vp(256), None, None)
    assert rc == G.GSPARC_ERR_TOO_LARGE
    rc = L.gsparc_bin_sort_noalloc(ctypes.byref(v), 100, vp(256), G.GSPARC_NOALLOC_MAX_PAIRS + 1,
                                   vp(256), None, vp(256), vp(256), None, None)
    assert rc == G.GSPARC_ERR_TOO_LARGE


def _sorted(r, n, cap, noalloc):
    keys = torch.empty(cap, dtype=torch.int64, device="cuda")
    ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    ranges = torch.empty((r.T, 2), dtype=torch.int32, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    if noalloc:
        G.gsparc_bin_sort_noalloc(r.view, n, r.proj, cap, ids, keys, ranges, npairs, status)
    else:
        G.gsparc_bin_sort(r.view, n, r.proj, cap, r.ws, ids, keys, ranges, npairs, status)
    assert G.gsparc_check(status) == 0
    m = int(npairs.item())
    return m, keys[:m].cpu(), ids[:m].cpu(), ranges.cpu()


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_two_calls_in_a_row():
    cap = G.GSPARC_NOALLOC_MAX_PAIRS
    # call 1: the 50,000-Gaussian scene projected on the GPU (about 395k pairs)
    sc = synth.make_scene(50_000, seed=0)
    r1 = Renderer(90, 360, 64, sc.n, pair_capacity=cap, device="cuda")
    ds = DeviceScene.from_host(sc, "cuda")
    G.gsparc_project(r1.view, ds.means, ds.log_scales, ds.quats, r1.proj)
    # call 2: a smaller, different problem on another grid (ragged tiles, six sort passes)
    rec = synth.make_proj_records(7001, 180, 720, seed=13)
    r2 = Renderer(180, 720, 1, rec.shape[0], pair_capacity=cap, device="cuda")
    r2.proj.copy_(torch.tensor(rec, device="cuda"))
    a1 = _sorted(r1, sc.n, cap, noalloc=True)
    a2 = _sorted(r2, rec.shape[0], cap, noalloc=True)
    b1 = _sorted(r1, sc.n, cap, noalloc=False)
    b2 = _sorted(r2, rec.shape[0], cap, noalloc=False)
    for a, b in ((a1, b1), (a2, b2)):
        assert a[0] == b[0] and a[0] > 0
        assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2]) and torch.equal(a[3], b[3])
    # and the first problem again after the second (leftover state must not leak)
    a3 = _sorted(r1, sc.n, cap, noalloc=True)
    assert a3[0] == b1[0]
    assert torch.equal(a3[1], b1[1]) and torch.equal(a3[2], b1[2]) and torch.equal(a3[3], b1[3])
