"""The warm-start network's GPU kernels against the FP64 reference, and what training gains."""
import numpy as np
import pytest

import workloads
from oracle.neural import bilinear_map, loss_and_grad
from paper_2305_09020_gb300 import native, warmstart

pytestmark = pytest.mark.gpu


def small_operator(seed=3):
    rng = np.random.default_rng(seed)
    dims = [3, 16, 24, 12 * 6]
    node_x = np.sort(rng.uniform(0.0, 2.0, 9))
    node_y = np.linspace(0.0, 1.0, 5)
    mean, std = np.array([1.5, 8.0, 0.1]), np.array([0.8, 5.0, 0.05])
    no = native.NeuralOperator(dims, mean, std, (12, 6), (0.0, 2.0, 0.0, 1.0), node_x, node_y, seed=seed)
    R = bilinear_map(12, 6, (0.0, 2.0, 0.0, 1.0), node_x, node_y)
    return no, dims, mean, std, R, rng


def test_gradients_match_fp64_reference():
    no, dims, mean, std, R, rng = small_operator()
    feat = np.column_stack([rng.uniform(0, 3, 8), rng.uniform(2, 20, 8), rng.uniform(0.03, 0.2, 8)])
    tgt = np.tanh(rng.standard_normal((8, R.shape[0])))
    loss, g = no.loss_grad(feat, tgt)
    p = no.params()
    lref, gref, pred = loss_and_grad(p, dims, mean, std, R, feat, tgt, bf16=True)
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    np.testing.assert_allclose(no.predict(feat), pred, atol=2e-6)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
    no.close()


def test_tensor_core_layers_match_fp64_reference():
    """Layer widths that run the hidden and output layers on the tensor cores (K = 64, 128, N = 128,
    256: tcgen05 kind::f16, BF16 weights, inputs split into BF16 head and tail, FP32 accumulation)
    and a batch of 80 (two 64-sample column blocks), against the FP64 reference: the inputs keep
    ~16 bits, so the predictions agree to 2e-5 and the gradients (CUDA-core backward) to 1e-4."""
    rng = np.random.default_rng(11)
    dims = [3, 64, 128, 16 * 16]
    node_x = np.sort(rng.uniform(0.0, 2.0, 13))
    node_y = np.linspace(0.0, 1.0, 7)
    mean, std = np.array([1.5, 8.0, 0.1]), np.array([0.8, 5.0, 0.05])
    no = native.NeuralOperator(dims, mean, std, (16, 16), (0.0, 2.0, 0.0, 1.0), node_x, node_y, seed=11)
    R = bilinear_map(16, 16, (0.0, 2.0, 0.0, 1.0), node_x, node_y)
    feat = np.column_stack([rng.uniform(0, 3, 80), rng.uniform(2, 20, 80), rng.uniform(0.03, 0.2, 80)])
    tgt = np.tanh(rng.standard_normal((80, R.shape[0])))
    loss, g = no.loss_grad(feat, tgt)
    lref, gref, pred = loss_and_grad(no.params(), dims, mean, std, R, feat, tgt, bf16=True)
    np.testing.assert_allclose(no.predict(feat), pred, atol=2e-5)
    assert abs(loss - lref) <= 1e-4 * abs(lref)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
    no.close()


def test_training_reduces_loss():
    no, dims, mean, std, R, rng = small_operator(seed=5)
    feat = np.column_stack([rng.uniform(0, 3, 64), rng.uniform(2, 20, 64), rng.uniform(0.03, 0.2, 64)])
    tgt = np.tanh(np.outer(feat[:, 0] - 1.5, np.linspace(-1, 1, R.shape[0])))
    losses = no.train(feat, tgt, batch=16, epochs=60, lr=3e-3, seed=1)
    assert losses[-1] < 0.2 * losses[0], losses[[0, -1]]
    no.close()


def test_warm_start_prediction_beats_cold_profile():
    """Trained on the states an ensemble reaches after 3000 steps, the network's field for held-out
    runs is closer to their state at that time than the usual initial profile is (coarse mesh)."""
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()

    def runs(n, seed):
        return workloads.warmstart2d(n, seed, 8, 4, 6)   # a coarse mesh so the test stays short

    train, test = runs(192, 101), runs(24, 202)
    f_tr, y_tr, _ = warmstart.generate(train, tol=0.0, max_steps=3000, check_every=3000, stream=s.cuda_stream)
    f_te, y_te, _ = warmstart.generate(test, tol=0.0, max_steps=3000, check_every=3000, stream=s.cuda_stream)
    no = warmstart.make_operator(f_tr, train[0].mesh, seed=0, stream=s.cuda_stream)
    no.train(f_tr, y_tr, batch=32, epochs=300, lr=1e-3, seed=0)
    pred = no.predict(f_te)
    x = native.nodes_1d(test[0].mesh.xb, 6, True)
    y = native.nodes_1d(test[0].mesh.yb, 6, False)
    cold = np.array([workloads.eval_on_grid(w.phi0, x, y, None).ravel() for w in test])
    e_warm = np.linalg.norm(pred - y_te, axis=1)
    e_cold = np.linalg.norm(cold - y_te, axis=1)
    assert np.median(e_warm) < np.median(e_cold), (np.median(e_warm), np.median(e_cold))
    no.close()


def test_warm_start_saves_steps_to_the_equilibrium():
    """The equilibrium system (Sec. 2.4) on a coarse mesh, FP64: trained on the equilibria of 256
    runs, the network's fields (shifted on the device to each run's phase mass) start 24 held-out
    runs that reach the pseudo-time criterion in fewer steps (median) than the same runs started
    cold; the judge is the cold start run to a tolerance ten times tighter.  Most warm runs end at
    the judge's equilibrium as closely as the cold runs do; some settle in another steady state,
    which the judge exposes (the cold start stays the fallback)."""
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()

    def runs(n, seed):
        return warmstart.equilibrium_runs(workloads.warmstart2d(n, seed, 8, 4, 6))

    tol, cap = 1e-3, 20000
    train, test = runs(256, 101), runs(24, 202)
    f_tr, y_tr, st_tr = warmstart.generate(train, tol=tol, max_steps=cap, check_every=500,
                                           precision=native.PF_FP64, stream=s.cuda_stream)
    assert (st_tr > 0).sum() > 200                        # the training targets are equilibria
    no = warmstart.make_operator(f_tr, train[0].mesh, seed=0, stream=s.cuda_stream)
    no.train(f_tr, y_tr, batch=32, epochs=600, lr=1e-3, seed=0)
    res = warmstart.evaluate(no, test, tol, cap, check_every=500, precision=native.PF_FP64,
                             stream=s.cuda_stream, judge_tol=tol / 10, judge_steps=4 * cap)
    no.close()
    cold, warm = res["cold"], res["warm"]
    assert warm["steps_median"] < 0.95 * cold["steps_median"], (warm["steps_median"], cold["steps_median"])
    ec, ew = np.array(cold["err"]), np.array(warm["err"])
    assert np.all(ec < 1e-3)                              # the criterion puts cold runs at the judge
    same = ew <= 3.0 * ec + 1e-4
    assert same.mean() >= 0.5, (ew, ec)
