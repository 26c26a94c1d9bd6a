"""The allocation-free entry point, for callers that cannot allocate device
memory (another component owns the allocator, or the memory budget is already
committed).  It must give the same result as the ordinary entry point, on two
calls in a row that share its fixed scratch array, also in a process that
never creates a context and with mass conservation in 3-D; reject arrays
whose scratch would not fit; and refuse stream capture.  This file is
collected last."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2609_34622_b300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda:0")


def test_noalloc_matches_context_entry_point_twice():
    import torch
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B
    B.build()
    torch.cuda.set_device(0)
    ctx = bm.Context(0)
    rng = np.random.default_rng(71)
    x1 = synth.ecg_signal(20000, 250.0, rng)
    y1, sp1 = synth.poisson_observe(x1, 50.0, rng)
    j2 = synth.config1()
    j3 = synth.config2()
    x4 = synth.texture_edge_image((512, 512), rng)
    y4, sp4 = synth.poisson_observe(x4, 5.0, rng)
    cases = [(y1, dict(noise=("poisson", sp1), patch=(32,), step=(4,), search=(129,), group_size=(16, 32))),
             (j2.y, j2.cfg), (j3.y, j3.cfg),
             (y4, dict(noise=("poisson", sp4), patch=(8, 8), step=(3, 3), search=(39, 39), group_size=(16, 32)))]
    for y, cfg in cases:
        ref = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
        ctx.bmnd_denoise(_cuda(y), ref, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"])
        refn = ref.cpu().numpy()
        for call in range(2):
            out = torch.full(y.shape, float("nan"), dtype=torch.float32, device="cuda:0")
            bm.bmnd_denoise_noalloc(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                                    cfg["group_size"])
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            PT.assert_voxels(got, refn, 1.0, what="noalloc call %d" % call)
    ctx.close()


def test_noalloc_rejects_arrays_beyond_its_scratch():
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y = torch.zeros(2048, 2048, device="cuda:0")
    out = torch.empty_like(y)
    with pytest.raises(bm.BmndError) as e:
        bm.bmnd_denoise_noalloc(y, out, ("gaussian", 0.1), (8, 8), (3, 3), (39, 39), (16, 32))
    assert e.value.status == bm.ENOMEM
    assert "scratch" in str(e.value)


def test_noalloc_3d_mass_conservation_twice():
    """24^3 Poisson volume, patch 4^3, step 2, search 11^3, both stages with
    mass conservation (the second sweep recomputes the filtering from the
    stored group tables, the path this entry point takes): equal to
    bmnd_denoise under the voxel contract, and sum(out) = sum(y), on two
    calls in a row."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    rng = np.random.default_rng(73)
    lam = synth.ellipsoid_phantom((24, 24, 24), rng)
    x = lam / lam.max()
    y, sp = synth.poisson_observe(x, 5.0, rng)
    cfg = dict(noise=("poisson", sp), patch=(4, 4, 4), step=(2, 2, 2), search=(11, 11, 11), group_size=(16, 32))
    ctx = bm.Context(0)
    ref = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), ref, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2, 3)
    refn = ref.cpu().numpy()
    ctx.close()
    for call in range(2):
        out = torch.full(y.shape, float("nan"), dtype=torch.float32, device="cuda:0")
        bm.bmnd_denoise_noalloc(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                                cfg["group_size"], 2, 3)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        PT.assert_voxels(got, refn, 1.0, what="noalloc 3-D mc call %d" % call)
        assert float(got.astype(np.float64).sum()) == pytest.approx(float(y.astype(np.float64).sum()), rel=1e-5)


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2609_34622_b300.bmnd as bm
from paper_2609_34622_b300 import synth
j = synth.config1()
torch.cuda.set_device(0)
y = torch.from_numpy(j.y).cuda()
out = torch.empty_like(y)
c = j.cfg
bm.bmnd_denoise_noalloc(y, out, c["noise"], c["patch"], c["step"], c["search"], c["group_size"])
np.save(sys.argv[2], out.cpu().numpy())
"""


def test_noalloc_in_a_process_without_context(tmp_path):
    """A process that never creates a context: the first call's own set-up
    must provide everything the kernels read (transform tables and the
    butterfly-DCT constants).  Its output equals bmnd_denoise's."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    dst = str(tmp_path / "fresh.npy")
    subprocess.run([sys.executable, "-c", _FRESH, root, dst], check=True, timeout=300)
    got = np.load(dst)
    j = synth.config1()
    ctx = bm.Context(0)
    ref = torch.empty(j.y.shape, dtype=torch.float32, device="cuda:0")
    c = j.cfg
    ctx.bmnd_denoise(_cuda(j.y), ref, c["noise"], c["patch"], c["step"], c["search"], c["group_size"])
    ctx.close()
    PT.assert_voxels(got, ref.cpu().numpy(), 1.0, what="fresh process")


def test_noalloc_refuses_stream_capture():
    """A call on a capturing stream returns EUNSUPPORTED before enqueueing
    anything (its job table lives on the caller's stack)."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y = _cuda(np.zeros((64, 64), np.float32))
    out = torch.empty_like(y)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=s):
        try:
            bm.bmnd_denoise_noalloc(y, out, ("gaussian", 0.1), (8, 8), (3, 3), (9, 9), (16, 32), stream=s)
        except bm.BmndError as e:
            status = e.status
    assert status == bm.EUNSUPPORTED
