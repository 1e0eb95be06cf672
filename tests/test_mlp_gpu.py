"""The proposal network's BF16 tensor-core forward/backward against the FP64
reference (oracle/mlp_ref.py) on the same bf16-rounded weights and inputs,
training progress, and the exactness of the learned Metropolis-Hastings
chains (they must still sample the Boltzmann weights of Sec. 3)."""
import numpy as np
import pytest

import oracle
from oracle import mlp_ref
import paper_1507_00315_gb300 as sk
from tests import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _flat(params):
    W1, b1, W2, b2, W3, b3 = params
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]).astype(np.float32)


def _unflat(v, n, nm):
    sizes = [(2 * n, 256), (256,), (256, 256), (256,), (256, nm), (nm,)]
    out, o = [], 0
    for s in sizes:
        c = int(np.prod(s))
        out.append(v[o:o + c].reshape(s).astype(np.float64))
        o += c
    return out


@pytest.mark.parametrize("tensor_memory", [True, False])
@pytest.mark.parametrize("variant,n", [(0, 8), (1, 12), (0, 33)])
def test_forward_matches_fp64(variant, n, tensor_memory):
    d = si.differences(variant, n)
    off, nslot = mlp_ref.move_table(n, d)
    nm = int(nslot.sum())
    model = sk.Mlp(variant, n, 512, seed=1)
    model.set_gemm(tensor_memory)
    assert model.n_moves == nm
    params = si.mlp_params(5, 2 * n, 256, nm)
    params = list(params)
    params[1], params[3], params[5] = [si.bf16_round(p) for p in (params[1], params[3], params[5])]
    model.set_params(_flat(params))
    slots = si.random_slots(7, 300, n, d)
    z = model.forward(slots)
    model.check()
    x = mlp_ref.occupancy(slots, n, d)
    _, _, _, _, zr = mlp_ref.forward(x, *params)
    err = np.abs(z - zr).max() / np.abs(zr).max()
    assert err < 2e-2, err


@pytest.mark.parametrize("tensor_memory", [True, False])
@pytest.mark.parametrize("variant,n,B", [(0, 8, 256), (1, 16, 256), (0, 20, 1024)])
def test_gradients_match_fp64(variant, n, B, tensor_memory):
    # both backward paths: tcgen05 (activation gradients with B streamed,
    # weight gradients from K-major copies with a fixed-order K split) and
    # mma.sync (split-K atomics); B = 1024 gives the tcgen05 weight gradients
    # a K split over 16 slices
    d = si.differences(variant, n)
    off, nslot = mlp_ref.move_table(n, d)
    nm = int(nslot.sum())
    model = sk.Mlp(variant, n, B, seed=2)
    model.set_gemm(tensor_memory)
    params = [si.bf16_round(p) for p in si.mlp_params(11, 2 * n, 256, nm)]
    model.set_params(_flat(params))
    slots = si.random_slots(13, B, n, d)
    loss, g = model.loss_grad(slots, beta_star=2.0)
    model.check()
    x = mlp_ref.occupancy(slots, n, d)
    mask = mlp_ref.valid_mask(slots, n, d)
    target = mlp_ref.target_distribution(slots, n, d, 2.0)
    lr, gr = mlp_ref.loss_and_grads(x, *params, mask, target)
    assert abs(loss - lr) / abs(lr) < 1e-2
    got = _unflat(g, n, nm)
    for name, a in zip(["W1", "b1", "W2", "b2", "W3", "b3"], got):
        ref = gr[name]
        rel = np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-12)
        assert rel < 3e-2, (name, rel)
    # round trip of the parameters
    assert np.array_equal(model.get_params(), _flat(params))


def test_training_lowers_the_loss():
    n, variant = 12, 0
    d = si.differences(variant, n)
    res = sk.pt_run(variant, n, np.linspace(0, 6, 16), 256, 300, 0, 5, want_final=True)
    states = res["final_slots"].reshape(-1, n)                 # 4096 states from plain PT
    model = sk.Mlp(variant, n, 1024, seed=3)
    l0, _ = model.loss_grad(states[:1024], 2.0)
    l1, ms = model.train(states, epochs=30, batch=1024, lr=2e-3, beta_star=2.0, seed=1)
    l2, _ = model.loss_grad(states[:1024], 2.0)
    assert l2 < l0 * 0.9, (l0, l1, l2)


@pytest.mark.parametrize("variant,n", [(0, 5), (1, 4)])
def test_learned_chains_are_exact(variant, n):
    # an untrained network: a poor proposal, so long equilibrated runs
    beta = np.array([0.0, 0.7, 1.5, 2.6, 4.0, 6.0, 9.0, 14.0])
    model = sk.Mlp(variant, n, 8192, seed=4)
    res = sk.pt_run(variant, n, beta, 1024, 20000, 10000, 21, model=model)
    N = oracle.simplified_energy_hist(variant, n).astype(np.float64)
    E = np.arange(2 * n + 1)
    for j in range(len(beta)):
        p = N * np.exp(-beta[j] * E)
        p /= p.sum()
        h = res["hist"][j].astype(np.float64)
        assert np.abs(h / h.sum() - p).max() < 0.01, (j, h / h.sum(), p)
    est = oracle.pt_estimate_from_hist(res["hist"], beta, variant, n)
    assert abs(est / (oracle.backtrack_count(variant, n) / 2) - 1) < 0.02


@pytest.mark.parametrize("variant,n", [(0, 5), (1, 4)])
def test_learned_chains_exact_when_the_row_maximum_underflows(variant, n):
    # Logits of -100 on every move (W3 = 0, b3 = -100) while the padding
    # columns inside the move table's last 8-move word stay 0 (n = 5 Skolem:
    # 35 moves, Langford n = 4: 18): the step kernel's unmasked shift, the
    # row's largest element, is then 0 and every valid weight e^-100
    # underflows, so it must take the valid moves' maximum instead.  The
    # proposal is uniform over the valid moves and the chains must still
    # sample the exact Boltzmann weights.
    d = si.differences(variant, n)
    _, nslot = mlp_ref.move_table(n, d)
    nm = int(nslot.sum())
    assert nm % 8
    rng = np.random.default_rng(5)
    params = [rng.normal(0.0, 0.1, (2 * n, 256)), np.zeros(256), rng.normal(0.0, 0.1, (256, 256)),
              np.zeros(256), np.zeros((256, nm)), np.full(nm, -100.0)]
    model = sk.Mlp(variant, n, 8192, seed=4)
    model.set_params(_flat(params))
    beta = np.array([0.0, 0.7, 1.5, 2.6, 4.0, 6.0, 9.0, 14.0])
    res = sk.pt_run(variant, n, beta, 1024, 20000, 10000, 23, model=model)
    model.check()
    model.close()
    N = oracle.simplified_energy_hist(variant, n).astype(np.float64)
    E = np.arange(2 * n + 1)
    for j in range(len(beta)):
        p = N * np.exp(-beta[j] * E)
        p /= p.sum()
        h = res["hist"][j].astype(np.float64)
        assert np.abs(h / h.sum() - p).max() < 0.01, (j, h / h.sum(), p)
    assert res["acc_move"].min() > 0


def _hot_energy_distribution(variant, n, samples, seed):
    # The energy (empty bins) of the simplified problem at beta = 0: every pair
    # at an independent uniform start slot, straight from the definition.
    d = si.differences(variant, n)
    rng = np.random.default_rng(seed)
    counts = np.zeros(2 * n + 1)
    chunk = 250_000
    rows = np.arange(chunk)
    for _ in range(samples // chunk):
        occ = np.zeros((chunk, 2 * n), np.int8)
        for dk in d:
            s = rng.integers(0, 2 * n - dk, chunk)
            occ[rows, s] += 1
            occ[rows, s + dk] += 1
        counts += np.bincount((occ == 0).sum(1), minlength=2 * n + 1)
    return counts / counts.sum()


@pytest.mark.parametrize("variant,n", [(0, 16), (0, 20), (1, 24)])
def test_learned_chains_sample_boltzmann_over_several_chunks(variant, n):
    # Move tables of 376, 590 and 828 moves: two, three and four 256-move
    # chunks a row (the draw's lane and chunk selection, reverse moves in
    # later chunks, rows staged in shared memory, the bound that rejects
    # without a row).  At the hot rungs P_beta(E) is proportional to
    # P_0(E) e^(-beta E), P_0 sampled from the definition (2e6 draws); an
    # untrained network proposes.
    p0 = _hot_energy_distribution(variant, n, 2_000_000, 17)
    beta = np.array([0.0, 0.3, 0.6, 1.0])
    model = sk.Mlp(variant, n, 4096 * 4, seed=3)
    res = sk.pt_run(variant, n, beta, 4096, 2000, 500, 31, model=model)
    model.check()
    model.close()
    E = np.arange(2 * n + 1)
    for j, b in enumerate(beta):
        p = p0 * np.exp(-b * E)
        p /= p.sum()
        h = res["hist"][j].astype(np.float64)
        assert np.abs(h / h.sum() - p).max() < 0.01, (j, np.abs(h / h.sum() - p).max())
    assert (res["acc_move"] > 0).all() and (res["acc_swap"][:-1] > 0).all()


@pytest.mark.parametrize("variant,n,batch", [(1, 20, 4096), (1, 20, 65536), (0, 24, 40000)])
def test_tensor_memory_and_mma_sync_paths_agree(variant, n, batch):
    # the two forward GEMM paths see the same bf16 operands; their fp32 sums
    # differ only in accumulation order.  65536 and 40000 states give every
    # CTA of the persistent tcgen05 GEMM several row tiles (the operand ring
    # and both tensor-memory accumulators wrap around); 40000 is ragged.
    d = si.differences(variant, n)
    model = sk.Mlp(variant, n, (batch + 127) // 128 * 128, seed=6)
    slots = si.random_slots(8, batch, n, d)
    model.set_gemm(True)
    a = model.forward(slots)
    model.check()
    model.set_gemm(False)
    b = model.forward(slots)
    assert np.abs(a - b).max() <= 1e-2 * np.abs(b).max()


@pytest.mark.parametrize("variant,n,batch", [(0, 20, 4096), (1, 20, 40000), (0, 12, 1024),
                                             (0, 24, 4096), (1, 40, 1024)])
def test_bf16_logits_of_the_chains(variant, n, batch):
    # The tempering chains read the logits rounded to bf16 from a forward that
    # stores only the move table's columns (the last column tile multiplies
    # that many, rounded up to 16, instead of 256).  Every logit must be the
    # fp32 forward's rounded to nearest: within half a bf16 step (2^-8
    # relative) plus a little for accumulation order, on both GEMM paths.
    # n = 20: 590 moves, a last tile of 80 columns; n = 24: 852 (96); n = 40:
    # 2380 (80); 40000 states: ragged, several row tiles per CTA.
    d = si.differences(variant, n)
    model = sk.Mlp(variant, n, (batch + 127) // 128 * 128, seed=9)
    slots = si.random_slots(12, batch, n, d)
    for tc in (True, False):
        model.set_gemm(tc)
        z = model.forward(slots).astype(np.float64)
        zb = (model.forward_bf16(slots).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        model.check()
        tol = 2.0 ** -8 * np.abs(z) + 1e-4 * np.abs(z).max()
        assert (np.abs(zb - z) <= tol).all(), (tc, float(np.abs(zb - z).max()))
        assert np.isfinite(zb).all()
    model.close()


@pytest.mark.parametrize("variant,n", [(0, 8), (1, 12)])
def test_training_steps_match_adam_in_fp64(variant, n):
    # Two sk_mlp_train steps on one fixed minibatch of 256 states (given
    # order, so each step sees exactly the batch sk_mlp_loss_grad sees; the
    # tcgen05 backward sums its K-split partials in a fixed order and 256 rows
    # take one column-sum block, so the GPU's gradient is the same bits in
    # both calls).  After each step the FP32
    # masters and both moments must equal mlp_ref.adam_step applied in FP64
    # to the pre-step state and that gradient, and the BF16 weight copies the
    # forward uses must be the masters rounded to nearest-even bf16 exactly.
    # The gradient itself is checked against the FP64 backward
    # (mlp_ref.loss_and_grads) at the bf16 tolerance of
    # test_gradients_match_fp64.
    d = si.differences(variant, n)
    _, nslot = mlp_ref.move_table(n, d)
    nm = int(nslot.sum())
    B, lr, beta_star = 256, 1e-3, 2.0
    model = sk.Mlp(variant, n, B, seed=2)
    params = [si.bf16_round(p) for p in si.mlp_params(17, 2 * n, 256, nm)]
    model.set_params(_flat(params))
    slots = si.random_slots(19, B, n, d)
    x = mlp_ref.occupancy(slots, n, d)
    mask = mlp_ref.valid_mask(slots, n, d)
    target = mlp_ref.target_distribution(slots, n, d, beta_star)
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    st0 = model.train_state()
    assert st0["t"] == 0 and not st0["m"].any() and not st0["v"].any()
    w = model.get_params().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for t in (1, 2):
        _, g = model.loss_grad(slots, beta_star)
        _, gr = mlp_ref.loss_and_grads(x, *_unflat(w, n, nm), mask, target)
        for name, a in zip(names, _unflat(g, n, nm)):
            rel = np.linalg.norm(a - gr[name]) / max(np.linalg.norm(gr[name]), 1e-12)
            assert rel < 3e-2, (t, name, rel)
        model.train(slots, epochs=1, batch=B, lr=lr, beta_star=beta_star, seed=sk.MLP_KEEP_ORDER)
        # the kernel's betas are the float32 values of 0.9 and 0.999
        # (0.999f is 1.3e-5 away from 0.999 in relative terms); the reference
        # takes the same two numbers
        w_ref, m_ref, v_ref = mlp_ref.adam_step(w, g.astype(np.float64), m, v, t, lr,
                                                b1=float(np.float32(0.9)),
                                                b2=float(np.float32(0.999)))
        w_gpu = model.get_params().astype(np.float64)
        st = model.train_state()
        assert st["t"] == t
        # FP32 arithmetic of one update: a few ulp of each moment (m can
        # cancel at t = 2, so its tolerance is scaled by the largest |m|).
        # The step lr * mhat / (sqrt(vhat) + eps) is at most lr here (by
        # Cauchy-Schwarz over the two gradients), and the host's fp32 bias
        # correction 1 - beta2^t is off by up to 2^-24 / (1 - beta2^t) =
        # 1.5e-5 relative at t = 2, 7.5e-6 of the step after the square root.
        assert np.allclose(st["m"], m_ref, rtol=1e-5, atol=1e-6 * np.abs(m_ref).max()), t
        assert np.allclose(st["v"], v_ref, rtol=1e-5, atol=1e-30), t
        err = np.abs(w_gpu - w_ref)
        tol = 2e-5 * lr + 2.0 ** -22 * np.abs(w_ref)
        assert (err <= tol).all(), (t, float(err.max()), int((err > tol).sum()))
        assert np.abs(w_gpu - w).max() > 0.5 * lr           # the step moved the weights
        used = _unflat(st["used"], n, nm)
        masters = _unflat(w_gpu, n, nm)
        for i, name in enumerate(names):
            want = si.bf16_round(masters[i]) if name.startswith("W") else masters[i]
            assert np.array_equal(used[i], want), (t, name)
        w, m, v = w_gpu, st["m"].astype(np.float64), st["v"].astype(np.float64)


def test_trained_network_gains_over_plain_tempering_per_iteration(skolem_table):
    # What the trained network gains over the method without it.  A network
    # trained on plain-tempering states proposes moves that the
    # Metropolis-Hastings test accepts far more often, and at equal
    # iterations its estimate of S(12) is far closer to the exact count
    # (Table 7) than the plain chains'.  On one GB300 (512 ladders, 3200
    # iterations, 10 % burn-in, six seeds each): plain -98.8 % (standard
    # error 0.04 %), learned -23 % (0.5 %); mid-ladder move acceptance 0.22
    # plain, 0.53 learned.  Per unit of GPU time the plain chains win: a
    # learned iteration runs the network over every proposed state.
    v, n, L, iters = 0, 12, 512, 3200
    beta = sk.tune_ladder(v, n, 32, 32.0, 0)
    states = np.concatenate([
        sk.pt_run(v, n, beta, 1024, 1000, 0, 100 + s, want_final=True)["final_slots"].reshape(-1, n)
        for s in range(8)])
    model = sk.Mlp(v, n, L * 32, seed=1)
    model.train(states, epochs=5, batch=4096, lr=1e-3, beta_star=2.0, seed=1)
    res = {}
    for name, mdl in (("plain", None), ("learned", model)):
        errs, acc = [], []
        for seed in range(6):
            r = sk.pt_run(v, n, beta, L, iters, iters // 10, 1000 + seed, model=mdl)
            est, _, _ = sk.pt_estimate_hist(v, n, beta, r["hist"])   # reflections identified
            errs.append(est / skolem_table[n] - 1)
            acc.append(float(r["acc_move"][16]) / (L * iters))
        res[name] = (float(np.mean(errs)), float(np.std(errs, ddof=1) / np.sqrt(len(errs))),
                     float(np.mean(acc)))
    model.close()
    (ep, sp, ap), (el, sl, al) = res["plain"], res["learned"]
    gain = abs(ep) - abs(el)
    assert gain > 0.3 and gain > 10 * np.hypot(sp, sl), res
    assert al > 1.5 * ap, res
