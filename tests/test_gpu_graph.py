"""The training step and the E/F/W + grade step captured in CUDA graphs (after one warm-up
call sizes the workspaces) and replayed: bitwise the eager results, also after new parameters
are loaded between replays (the kernels read the parameters from the model's device buffer)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2304_13144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api(native_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_13144_gb300 import api as A
    return A


def theta_for(md, seed):
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    return synth.draw_theta(seed, md.n_types, md.n_rad, md.n_q, nu_sum, nf, md.r_min, md.r_cut, 40.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_train_step_graph_replay(api, prec):
    md = O.OracleModel(3, 16, 2.0, 5.0)
    th0, th1 = theta_for(md, 91), theta_for(md, 92)
    bnp = synth.training_batch(seed=93, n_cfg=64, n_types=3, lo=8, hi=64)
    model = api.mtp_load(api.make_desc(3, 16), th0)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    g = synth.rng(94)
    E = torch.tensor(g.normal(size=b.n_cfg), device="cuda")
    F = torch.tensor(g.normal(scale=0.05, size=(b.n_atoms, 3)), device="cuda")
    Wr = torch.tensor(g.normal(scale=0.5, size=(b.n_cfg, 9)), device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(model.n_params, dtype=torch.float64, device="cuda")

    def step():
        api._check(api.lib().mtp_train_step(model.h, api.ctypes.byref(b.c), nb.h, api._prec(prec), api._ptr(E),
                                            api._ptr(F), api._ptr(Wr), 1.0, 0.01, 0.001, api._ptr(loss),
                                            api._ptr(grad), api._stream()))

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()                                   # warm-up: sizes every workspace
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager0 = (loss.clone(), grad.clone())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(loss, eager0[0]) and torch.equal(grad, eager0[1])
    api.mtp_set_params(model, th1)
    step()
    torch.cuda.synchronize()
    eager1 = (loss.clone(), grad.clone())
    api.mtp_set_params(model, th0)
    api.mtp_set_params(model, th1)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(loss, eager1[0]) and torch.equal(grad, eager1[1])
    assert not torch.equal(eager0[1], eager1[1])


def test_md_step_graph_replay(api):
    md = O.OracleModel(3, 20, 2.0, 5.0)
    theta = theta_for(md, 95)
    model = api.mtp_load(api.make_desc(3, 20), theta)
    api.mtp_set_active_set(model, torch.tensor(synth.diag_dominant(96, md.m), device="cuda"))
    bnp = synth.fcc_ternary(seed=97, n=10)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(model, b)
    out = api.mtp_step(model, b, nb, "mixed")                     # warm-up, allocates outputs
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in out.items() if v is not None}
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.mtp_step(model, b, nb, "mixed", out=out)
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(graph):
        api.mtp_step(model, b, nb, "mixed", out=out)
    for v in out.values():
        if v is not None:
            v.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for k, v in eager.items():
        assert torch.equal(out[k], v), k
