"""Batches: many trees (different kernels, alpha, p, depth) in one CUDA graph give the same bits as
evaluating each tree alone, and match the oracle."""
import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import inputs as I
from gpu_util import TOL_FP64, TOL_SPLIT, oracle_eval, rel_err, sample_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    V.load_library()


def _workloads():
    rng = np.random.default_rng(44)
    ws = []
    for k, (kernel, alpha, p) in enumerate([(0, 10.0, 8), (1, 30.0, 12), (0, 300.0, 16), (1, 1000.0, 8),
                                            (0, 55.0, 12), (1, 120.0, 16)]):
        tree = I.random_balanced_tree(rng, 10 + 5 * k, 6, side=2.0, min_depth=1)
        X, Y = I.node_coords(tree, p)
        fn = I.gaussian_sum(rng.uniform(-0.6, 0.6, (3, 2)), rng.uniform(0.1, 0.3, 3), rng.uniform(-1, 1, 3))
        ws.append(I.Workload(f"b{k}", kernel, alpha, p, tree, fn(X, Y)))
    return ws


@pytest.mark.parametrize("precision,engine", [(V.VP_PREC_FP64, None), (V.VP_PREC_SPLIT, None),
                                              (V.VP_PREC_SPLIT, V.ENGINE_TCGEN05)])
def test_batch_graph_matches_single_tree_evaluations(precision, engine):
    import torch
    ws = _workloads()
    vps = [V.VolumePotential(w.kernel, w.alpha, w.p, w.tree, precision=precision) for w in ws]
    try:
        if engine is not None:
            for vp in vps:
                V.vp_tree_set_engine(vp.tree, engine)
        fs = [torch.from_numpy(w.f).cuda() for w in ws]
        singles = [vp(f) for vp, f in zip(vps, fs)]
        us = [torch.full_like(f, float("nan")) for f in fs]
        gs = [torch.full((2, f.numel()), float("nan"), dtype=torch.float64, device="cuda") for f in fs]
        b = V.vp_batch_create([vp.tree for vp in vps], fs, us, gs, n_streams=4)
        try:
            for _ in range(2):   # the graph can be replayed
                V.vp_batch_run(b)
                torch.cuda.synchronize()
                for (u1, g1), u2, g2 in zip(singles, us, gs):
                    assert torch.equal(u1, u2) and torch.equal(g1, g2)
            nodes, launches = V.vp_batch_stats(b)
            assert nodes == sum(w.n_nodes for w in ws) and launches > len(ws)
        finally:
            V.vp_batch_free(b)
        # one-shot form, with and without a graph
        for use_graph in (0, 1):
            u3 = [torch.zeros_like(f) for f in fs]
            g3 = [torch.zeros(2, f.numel(), dtype=torch.float64, device="cuda") for f in fs]
            V.vp_eval_batched([vp.tree for vp in vps], fs, u3, g3, use_graph=use_graph)
            torch.cuda.synchronize()
            for (u1, _), u2 in zip(singles, u3):
                assert torch.equal(u1, u2)
        # against the oracle on sampled nodes
        tol = TOL_FP64 if precision == V.VP_PREC_FP64 else TOL_SPLIT
        for w, (u1, g1) in zip(ws, singles):
            idx = sample_nodes(w, 60, 5)
            ou, oux, ouy = oracle_eval(w, idx)
            u1 = u1.cpu().numpy(); g1 = g1.cpu().numpy()
            errs = (rel_err(u1[idx], ou), rel_err(g1[0, idx], oux), rel_err(g1[1, idx], ouy))
            assert max(errs) < tol, (w.name, errs)
    finally:
        for vp in vps:
            vp.close()
