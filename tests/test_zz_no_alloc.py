"""sgs_densify_split_noalloc: the densify step for callers that cannot give the
library a workspace (code where cudaMalloc is not allowed or would stall the
device, or hosts that own every device allocation).  Its scratch is a fixed
array inside the library; this test checks, through the C ABI, that two calls
in a row give the same results as the workspace entry point, that the
largest allowed size with every scratch region in use (7-D eigenpairs held in
the scratch, the increment budget) does too, and that sizes beyond the
array's limit are refused before anything runs."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_2505_05587_gb300 import binding as B  # noqa: E402
from paper_2505_05587_gb300 import pipeline as PL  # noqa: E402


def _inputs(seed, n, sh_degree):
    scene = synth.cluster_scene(seed, n, sh_degree)
    g = B.GaussianTensors.from_scene(scene)
    rng = np.random.default_rng(seed + 100)
    S = torch.as_tensor(rng.normal(0.0, 1e-2, (n, 6)).astype(np.float32)).cuda()
    gn = torch.as_tensor(rng.uniform(0.0, 1.0, n).astype(np.float32)).cuda()
    return g, S, gn


def _run(fn_noalloc, g, S, gn, eps_split, step_scale, inv_T):
    db = PL.DensifyBuffers.alloc(g)
    if fn_noalloc:
        B.densify_split_noalloc(g, S, inv_T, eps_split, step_scale, gn, 0.5, db.out, db.capacity, db.n_out,
                                db.parent, db.lam, db.v)
    else:
        B.densify_split(g, S, inv_T, eps_split, step_scale, gn, 0.5, db.out, db.capacity, db.n_out, db.parent,
                        db.lam, db.v, db.split_ws)
    torch.cuda.synchronize()
    return db


def _compare(a, b, S, inv_T):
    n_out = int(a.n_out.item())
    assert int(b.n_out.item()) == n_out
    assert torch.equal(a.parent[:n_out], b.parent[:n_out])
    nrm = torch.linalg.norm(S, dim=1) * inv_T
    assert bool(torch.all((a.lam - b.lam).abs() <= 1e-4 * nrm.clamp_min(1e-30)))
    assert float((a.out.means[:n_out] - b.out.means[:n_out]).abs().max()) <= 1e-6
    assert float((a.out.opacity_logit[:n_out] - b.out.opacity_logit[:n_out]).abs().max()) <= 1e-5
    for f in ("log_scales", "quats", "sh"):
        assert torch.equal(getattr(a.out, f)[:n_out], getattr(b.out, f)[:n_out])


def test_noalloc_matches_workspace_entry_point_two_calls():
    # first call: larger scene, SH degree 3, gradient gate on
    g1, S1, gn1 = _inputs(0, 20000, 3)
    ref1 = _run(False, g1, S1, gn1, 0.0, 1.0, 1.0)
    got1 = _run(True, g1, S1, gn1, 0.0, 1.0, 1.0)
    _compare(ref1, got1, S1, 1.0)
    # second call in a row: smaller scene, other degree and thresholds (the
    # shared scratch still holds the first call's contents)
    g2, S2, gn2 = _inputs(1, 7001, 1)
    ref2 = _run(False, g2, S2, gn2, -1e-6, 0.5, 0.25)
    got2 = _run(True, g2, S2, gn2, -1e-6, 0.5, 0.25)
    _compare(ref2, got2, S2, 0.25)
    assert int(got1.n_out.item()) > g1.n and int(got2.n_out.item()) > g2.n


def _split_both(g, S, eps_split, step, budget, S_po=None, S_ls=None, eig_out=True):
    """The workspace entry point and the allocation-free one on the same inputs."""
    dim = 3 if S_po is None else (4 if S_ls is None else 7)
    res = []
    for noalloc in (False, True):
        db = PL.DensifyBuffers.alloc(g, dim_theta=dim)
        lam, v = (db.lam, db.v) if eig_out else (None, None)
        if noalloc:
            B.densify_split_noalloc(g, S, 1.0, eps_split, step, None, 0.0, db.out, db.capacity, db.n_out, db.parent,
                                    lam, v, max_splits=budget, S_po=S_po, S_ls=S_ls)
        else:
            B.densify_split(g, S, 1.0, eps_split, step, None, 0.0, db.out, db.capacity, db.n_out, db.parent, lam,
                            v, db.split_ws, max_splits=budget, S_po=S_po, S_ls=S_ls)
        torch.cuda.synchronize()
        res.append(db)
    return res


def _same_split(a, b):
    n_out = int(a.n_out.item())
    assert int(b.n_out.item()) == n_out
    assert torch.equal(a.parent[:n_out], b.parent[:n_out])
    for f in ("means", "log_scales", "opacity_logit"):
        assert float((getattr(a.out, f)[:n_out] - getattr(b.out, f)[:n_out]).abs().max()) <= 1e-6, f
    for f in ("quats", "sh"):
        assert torch.equal(getattr(a.out, f)[:n_out], getattr(b.out, f)[:n_out])
    return n_out


def test_noalloc_largest_size_theta7_budget_scratch_eigenpairs():
    """The worst case of the fixed scratch: n at its limit (1,000,000), the
    7-component eigenvectors and the eigenvalues kept in the scratch (no
    caller outputs for them), and the increment budget's tie flags and select
    state in use."""
    n = 1_000_000
    g, S, _ = _inputs(2, n, 0)
    rng = np.random.default_rng(5)
    S_po = torch.as_tensor(rng.normal(0.0, 1e-2, (n, 3)).astype(np.float32)).cuda()
    S_ls = torch.as_tensor(rng.normal(0.0, 1e-2, (n, 18)).astype(np.float32)).cuda()
    a, b = _split_both(g, S, 0.0, 0.5, 4096, S_po=S_po, S_ls=S_ls, eig_out=False)
    assert _same_split(a, b) == n + 4096


def test_noalloc_theta4_with_budget_and_eigen_outputs():
    g, S, _ = _inputs(3, 30000, 2)
    rng = np.random.default_rng(6)
    S_po = torch.as_tensor(rng.normal(0.0, 1e-2, (g.n, 3)).astype(np.float32)).cuda()
    a, b = _split_both(g, S, -1e-6, 0.3, 1000, S_po=S_po)
    assert _same_split(a, b) == g.n + 1000
    assert torch.equal(a.lam, b.lam) and torch.equal(a.v, b.v)


def test_noalloc_refuses_sizes_beyond_its_scratch():
    n = 1_000_001                       # buffers really hold n rows
    g = B.GaussianTensors.empty(n, 0)
    for t in g.tensors():
        t.zero_()
    S = torch.zeros(n, 6, device="cuda")
    out = B.GaussianTensors.empty(2 * n, 0)   # in bounds even if the call went ahead
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(B.SteepGSError) as e:
        B.densify_split_noalloc(g, S, 1.0, 0.0, 1.0, None, 0.0, out, 2 * n, n_out, None, None, None)
    assert e.value.status == 1
    torch.cuda.synchronize()
    assert int(n_out.item()) == 0
