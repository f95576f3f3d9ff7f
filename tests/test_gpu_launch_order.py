"""Kernels are launched with programmatic dependent launch (each kernel waits
for its predecessor's grid before it touches memory).  The results must not
depend on it: the same spatial and tonal optimisation with the attribute
switched off (FEM_PDL=0, plain stream order, in a child process) gives the
same mesh bit for bit and the same tonal values to rounding."""
import os
import subprocess
import sys

import numpy as np
import pytest

import seeded_inputs as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import seeded_inputs as S
import paper_2105_01586_gb300 as fem
n, dens, frac, out = {n}, {dens}, {frac}, {out!r}
f = torch.from_numpy(S.make_image(n, 3)).cuda()
m = fem.Mesh(n)
m.spatial_refine(f, dens, fem.params(topk_frac=frac))
g = m.tonal_opt(f)
xy, tri, mk = m.export()
np.savez(out, xy=xy, tri=tri, mk=mk, g=g.cpu().numpy())
"""


def _run(fem, n, dens, frac):
    f = torch.from_numpy(S.make_image(n, 3)).cuda()
    m = fem.Mesh(n)
    m.spatial_refine(f, dens, fem.params(topk_frac=frac))
    g = m.tonal_opt(f)
    xy, tri, mk = m.export()
    return xy, tri, mk, g.cpu().numpy()


@pytest.mark.parametrize("n,dens,frac", [(257, 0.04, 0.01), (513, 0.03, 0.01)])
def test_same_results_without_programmatic_launch(tmp_path, n, dens, frac):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_01586_gb300 as fem
    out = str(tmp_path / "plain.npz")
    env = dict(os.environ, FEM_PDL="0")
    subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, n=n, dens=dens, frac=frac, out=out)],
                   check=True, env=env, cwd=ROOT, timeout=300)
    ref = np.load(out)
    xy, tri, mk, g = _run(fem, n, dens, frac)
    assert np.array_equal(xy, ref["xy"]) and np.array_equal(tri, ref["tri"]) and np.array_equal(mk, ref["mk"])
    assert g.shape == ref["g"].shape
    np.testing.assert_allclose(g, ref["g"], rtol=0, atol=1e-6)
