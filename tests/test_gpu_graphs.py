"""Graph replay of the operators (cpct_plan_set_graphs).

In graph mode radon_fwd / radon_adj capture their kernels once per set of
buffer addresses and replay the CUDA graph afterwards.  The replay runs the
same kernels with the same arguments, so every result must equal the direct
launches bit for bit; profiling and the launch counter must see the same
kernels; changing the launch configuration must drop the graphs.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build
    build.build()
    return torch


def _inputs(torch, n, m, seed):
    rng = np.random.default_rng(seed)
    img = torch.from_numpy(rng.standard_normal((n, n)).astype(np.float32)).cuda()
    w = torch.from_numpy(rng.standard_normal((m, n)).astype(np.float32)).cuda()
    return img, w


@pytest.mark.parametrize("n,m,bins", [(256, 64, None), (512, 90, "quadtree"), (2048, 1024, None)])
def test_graph_replay_equals_direct_launches(torch_cuda, n, m, bins):
    torch = torch_cuda
    from paper_1009_1380_gb300.cpct import Plan
    img, w = _inputs(torch, n, m, n + m)
    direct = Plan(n, n, m)
    graphed = Plan(n, n, m)
    if bins:
        # bins of several sizes: the capture forks onto the plan's side streams
        for p in (direct, graphed):
            p.set_bins("fwd", bins)
            p.set_bins("adj", bins)
    graphed.set_graphs(True)
    y0 = direct.fwd(img)
    z0 = direct.adj(w)
    y1 = torch.empty_like(y0)
    z1 = torch.empty_like(z0)
    direct.launch_count(reset=True)
    graphed.launch_count(reset=True)
    for rep in range(3):
        y1.fill_(float("nan"))
        z1.fill_(float("nan"))
        graphed.fwd(img, y1)
        graphed.adj(w, z1)
        torch.cuda.synchronize()
        assert torch.equal(y0, y1), rep
        assert torch.equal(z0, z1), rep
    assert graphed.graphs() == 2
    direct.fwd(img, y0)
    direct.adj(w, z0)
    # one application's kernels counted per replay
    assert graphed.launch_count() == 3 * direct.launch_count()
    direct.sync()
    graphed.sync()


def test_graphs_follow_addresses_and_configuration(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300.cpct import Plan
    n, m = 256, 48
    img, w = _inputs(torch, n, m, 7)
    p = Plan(n, n, m)
    p.set_graphs(True)
    outs = [torch.empty((m, n), device="cuda") for _ in range(10)]
    for o in outs:
        p.fwd(img, o)
    # at most 8 graphs are kept
    assert p.graphs() == 8
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    # a new work-item cap drops the graphs; results follow the new plan
    p.set_caps(fwd_cap=300, adj_cap=12)
    assert p.graphs() == 0
    ref = Plan(n, n, m)
    ref.set_caps(fwd_cap=300, adj_cap=12)
    z_ref = ref.adj(w)
    z = torch.empty_like(z_ref)
    p.adj(w, z)
    p.adj(w, z)
    torch.cuda.synchronize()
    assert p.graphs() == 1
    assert torch.equal(z, z_ref)
    p.set_graphs(False)
    assert p.graphs() == 0
    p.sync()
    ref.sync()


def test_profiling_inside_graphs(torch_cuda):
    """Profiled kernels keep their event brackets in graph mode: every replay
    records its own pair of events."""
    torch = torch_cuda
    from paper_1009_1380_gb300.cpct import Plan
    n, m = 512, 128
    img, _ = _inputs(torch, n, m, 11)
    p = Plan(n, n, m)
    p.set_graphs(True)
    y = torch.empty((m, n), device="cuda")
    z = torch.empty((n, n), device="cuda")
    p.profile_enable(0x1FF)
    for _ in range(4):
        p.fwd(img, y)
        p.adj(y, z)
    torch.cuda.synchronize()
    prof = p.profile_read()
    p.profile_enable(0)
    for name in ("k_fwd_col", "k_fwd_row", "k_fwd_interp", "k_fwd_ray", "k_adj_ray", "k_adj_spread",
                 "k_adj_row", "k_adj_col"):
        ms, cnt = prof[name]
        assert cnt == 4 and ms > 0.0, (name, prof[name])
    p.sync()


def test_calls_inside_a_caller_capture_launch_directly(torch_cuda):
    """A call made while the caller's stream is being captured lands in the
    caller's graph (no nested capture); replaying that graph gives the
    direct result."""
    torch = torch_cuda
    from paper_1009_1380_gb300.cpct import Plan
    n, m = 256, 64
    img, _ = _inputs(torch, n, m, 3)
    p = Plan(n, n, m)
    y0 = p.fwd(img)
    p.set_graphs(True)
    y = torch.empty_like(y0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.fwd(img, y)  # warm-up outside capture (captures the plan's own graph)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        p.fwd(img, y)
    y.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, y0)
    p.sync()


def test_host_buffer_operators_in_graph_mode(torch_cuda):
    """radon_fwd_host / radon_adj_host replay their graphs (the plan's staging
    buffers are the same on every call) and give the device operators'
    results bit for bit, call after call."""
    torch = torch_cuda
    from paper_1009_1380_gb300.cpct import Plan
    n, m = 256, 90
    rng = np.random.default_rng(5)
    p = Plan(n, n, m)
    imgs = [rng.standard_normal((n, n)).astype(np.float32) for _ in range(3)]
    ref = [(p.fwd(torch.from_numpy(im).cuda()).cpu().numpy(),) for im in imgs]
    ref = [(y, p.adj(torch.from_numpy(y).cuda()).cpu().numpy()) for (y,) in ref]
    p.set_graphs(True)
    for k in range(2):
        for im, (y_ref, z_ref) in zip(imgs, ref):
            y = p.fwd_host(im)
            z = p.adj_host(y)
            np.testing.assert_array_equal(y, y_ref)
            np.testing.assert_array_equal(z, z_ref)
    assert p.graphs() == 2
    p.sync()
