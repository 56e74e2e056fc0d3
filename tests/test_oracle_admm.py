"""Pins of the oracle's ADMM pieces: x-step penalty (Eq. 7, 8a, 12a), Adam,
consensus and dual update (Eq. 8b-c, 12b-c), over-relaxation (Sec. 3.3),
residuals (Eq. 9), the zero-mean dual invariant (Appendix, proof of Eq. 8b)
and textbook convergence of consensus ADMM on quadratics."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def tiny_layout(x_vals, u_vals, z_prev, deg=0):
    """One global Gaussian held by len(x_vals) blocks; every parameter of
    copy k equals x_vals[k]."""
    P = 11 + 3 * (deg + 1) ** 2
    n = len(x_vals)
    x = np.repeat(np.asarray(x_vals, np.float64)[:, None], P, 1).copy()
    u = np.repeat(np.asarray(u_vals, np.float64)[:, None], P, 1).copy()
    z = np.full((1, P), float(z_prev))
    return x, u, z, np.array([0, n], np.int64), np.arange(n, dtype=np.int32)


def test_hand_worked_consensus(oracle):
    cases = json.load(open(os.path.join(GOLD, "admm_two_block.json")))["cases"]
    for c in cases:
        x, u, z, off, cp = tiny_layout(c["x"], c["u"], c["z_prev"])
        oracle.consensus(x, u, z, off, cp, 0, alpha=c["alpha"])
        np.testing.assert_allclose(z, c["z"], rtol=0, atol=1e-15, err_msg=c["name"])
        np.testing.assert_allclose(u[:, 0], c["u_new"], atol=1e-15, err_msg=c["name"])
        np.testing.assert_allclose(u, np.repeat(np.asarray(c["u_new"])[:, None], u.shape[1], 1), atol=1e-15)


def test_unshared_global_copies_x(oracle):
    x, u, z, off, cp = tiny_layout([5.0], [0.0], -1.0)
    oracle.consensus(x, u, z, off, cp, 0, alpha=1.7)
    np.testing.assert_array_equal(z, 5.0)
    np.testing.assert_array_equal(u, 0.0)


def random_sharing(rng, n_glob, K):
    """Each global held by 1..4 of K blocks; copies laid out block by block."""
    members = [np.sort(rng.choice(K, rng.integers(1, min(4, K) + 1), replace=False)) for _ in range(n_glob)]
    copies = [(k, i) for k in range(K) for i in range(n_glob) if k in members[i]]
    gid = np.array([i for _, i in copies], np.int32)
    order = np.argsort(gid, kind="stable")
    off = np.concatenate([[0], np.cumsum(np.bincount(gid, minlength=n_glob))]).astype(np.int64)
    return gid, off, order.astype(np.int32)


def test_dual_mean_is_zero_after_consensus_and_full_equals_simplified(oracle):
    """Appendix: averaging Eq. 8c over the blocks gives u_bar = 0 after every
    consensus, so afterwards z = mean(x + u) equals z = mean(x)."""
    O = oracle
    rng = np.random.default_rng(0)
    gid, off, cp = random_sharing(rng, 40, 4)
    P = 14
    x = rng.standard_normal((len(gid), P))
    u = rng.standard_normal((len(gid), P))
    z = rng.standard_normal((40, P))
    for alpha in (1.0, 1.6):
        uu, zz = u.copy(), z.copy()
        O.consensus(x, uu, zz, off, cp, 0, alpha=alpha)
        shared = np.diff(off) > 1
        for i in np.nonzero(shared)[0]:
            np.testing.assert_allclose(uu[cp[off[i]:off[i + 1]]].mean(0), 0.0, atol=1e-14)
        # next round: complete form vs the simplified z = mean(x) (alpha = 1)
        x2 = x + rng.standard_normal(x.shape)
        zfull = zz.copy(); u2 = uu.copy()
        O.consensus(x2, u2, zfull, off, cp, 0, alpha=1.0)
        for i in np.nonzero(shared)[0]:
            np.testing.assert_allclose(zfull[i], x2[cp[off[i]:off[i + 1]]].mean(0), atol=1e-13)


def test_residuals(oracle):
    x, u, z, off, cp = tiny_layout([1.0, 3.0], [0.0, 0.0], 0.5)
    rho = [2.0, 3.0, 4.0, 5.0, 6.0]
    res = oracle.consensus(x, u, z, off, cp, 0, alpha=1.0, rho=rho)
    # per parameter: ||x - z||^2 = 1 + 1; dual rho^2 * n * (2 - 0.5)^2
    counts = [3, 4, 3, 3, 1]          # mean, quat, scale, SH(deg 0), opacity
    for gi, c in enumerate(counts):
        assert res[gi] == pytest.approx(2.0 * c)
        assert res[5 + gi] == pytest.approx(rho[gi] ** 2 * 2 * 1.5 ** 2 * c)


def test_scaled_form_identity():
    """Appendix derivation of Eq. 7 (its middle line is garbled in the text;
    the identity it reaches): y.r + rho/2 ||r||^2 = rho/2 ||r + u||^2 - rho/2 ||u||^2
    with u = y / rho."""
    rng = np.random.default_rng(1)
    for _ in range(100):
        y, r = rng.standard_normal(7), rng.standard_normal(7)
        rho = rng.uniform(1e-3, 1e4)
        u = y / rho
        lhs = y @ r + rho / 2 * r @ r
        rhs = rho / 2 * (r + u) @ (r + u) - rho / 2 * u @ u
        assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-10 * rho)


def adam_case(oracle, step, g_loss, x0, z0, u0, shared, m0=0.0, v0=0.0):
    P = 14
    x = np.full((1, P), x0); g = np.full((1, P), g_loss)
    m = np.full((1, P), m0); v = np.full((1, P), v0)
    z = np.full((1, P), z0); u = np.full((1, P), u0)
    rho = np.array([10.0, 20.0, 30.0, 40.0, 50.0])
    lr = np.array([1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3])
    oracle.adam_admm_step(x, g, m, v, z, u, np.zeros(1, np.int32), np.array([shared], np.uint8),
                          rho, lr, 0, b1=0.9, b2=0.999, eps=1e-15, step=step)
    return x, m, v, rho, lr


def test_adam_penalty_first_step_closed_form(oracle):
    """Step 1: m_hat = g, v_hat = g^2, so x1 = x0 - lr g / (|g| + eps), with
    g = dL/dx + rho_grp (x0 - z + u) on a shared copy."""
    x, m, v, rho, lr = adam_case(oracle, 1, 0.25, 1.0, 0.4, 0.1, 1)
    grp = [0] * 3 + [1] * 4 + [2] * 3 + [3] * 3 + [4]
    slot = [0] * 3 + [1] * 4 + [2] * 3 + [3] * 3 + [5]
    for j in range(14):
        g = 0.25 + rho[grp[j]] * (1.0 - 0.4 + 0.1)
        assert x[0, j] == pytest.approx(1.0 - lr[slot[j]] * g / (abs(g) + 1e-15), rel=1e-14)
        assert m[0, j] == pytest.approx(0.1 * g)
        assert v[0, j] == pytest.approx(0.001 * g * g)
    # unshared copy: no penalty
    x, m, v, rho, lr = adam_case(oracle, 1, -0.5, 1.0, 0.4, 0.1, 0)
    np.testing.assert_allclose(x[0, :3], 1.0 + lr[0], rtol=1e-14)


def test_adam_second_step_closed_form(oracle):
    g, m0, v0, t = 0.3, 0.05, 0.002, 2
    x, m, v, rho, lr = adam_case(oracle, t, g, 2.0, 0.0, 0.0, 0, m0=m0, v0=v0)
    mm = 0.9 * m0 + 0.1 * g
    vv = 0.999 * v0 + 0.001 * g * g
    want = 2.0 - lr[0] * (mm / (1 - 0.9 ** t)) / (np.sqrt(vv / (1 - 0.999 ** t)) + 1e-15)
    assert x[0, 0] == pytest.approx(want, rel=1e-14)


def test_consensus_admm_on_quadratics_converges(oracle):
    """f_k(x) = a_k/2 ||x - b_k||^2 with the exact x-step
    x_k = (a_k b_k + rho (z - u_k)) / (a_k + rho) reaches the consensus
    optimum sum_k a_k b_k / sum_k a_k (Boyd et al., consensus ADMM)."""
    O = oracle
    rng = np.random.default_rng(2)
    K, P = 4, 14
    a = rng.uniform(0.5, 3.0, (K, 1))
    b = rng.standard_normal((K, P))
    x = np.zeros((K, P)); u = np.zeros((K, P)); z = np.zeros((1, P))
    off = np.array([0, K], np.int64); cp = np.arange(K, dtype=np.int32)
    rho = 1.0
    for alpha in (1.0, 1.6):
        x[:] = 0; u[:] = 0; z[:] = 0
        for _ in range(300):
            x[:] = (a * b + rho * (z - u)) / (a + rho)
            O.consensus(x, u, z, off, cp, 0, alpha=alpha)
        np.testing.assert_allclose(z[0], (a * b).sum(0) / a.sum(), atol=1e-10)


def test_adaptive_penalty_rule(oracle):
    """Eq. 10 on hand cases: r >> s doubles rho, s >> r halves it, balanced
    keeps it, nothing changes from iteration 2000 on."""
    rho = [1.0, 2.0, 3.0, 4.0, 5.0]
    res = [100.0, 1.0, 4.0, 0.0, 1e-6] + [0.01, 1.0, 1e-2 * 4.0 * 99, 4.0, 1.0]
    # group 0: r=10, s=0.1 -> inc; group 1: r=1, s=1 -> keep; group 2: r=2, s~1.99 -> keep;
    # group 3: r=0, s=2 -> dec; group 4: r=1e-3, s=1 -> dec
    assert oracle.adaptive_rho(rho, res, 10) == [2.0, 2.0, 3.0, 2.0, 2.5]
    assert oracle.adaptive_rho(rho, res, 2000) == rho


def test_dual_rescale_keeps_unscaled_dual(oracle):
    """u = y / rho: after rho changes and u is rescaled by rho_old / rho_new,
    the unscaled dual y = rho u is unchanged (Sec. 3.2, scaled form)."""
    rng = np.random.default_rng(5)
    P = 14
    u = rng.standard_normal((6, P))
    shared = np.array([1, 0, 1, 1, 0, 1], np.uint8)
    old = [1.0, 2.0, 3.0, 4.0, 5.0]
    new = [2.0, 2.0, 1.5, 8.0, 5.0]
    grp = [0] * 3 + [1] * 4 + [2] * 3 + [3] * 3 + [4]
    y_before = u * np.array([old[g] for g in grp])
    u2 = u.copy()
    oracle.scale_duals(u2, shared, [o / n for o, n in zip(old, new)], 0)
    y_after = u2 * np.array([new[g] for g in grp])
    np.testing.assert_allclose(y_after[shared == 1], y_before[shared == 1], rtol=1e-14)
    np.testing.assert_array_equal(u2[shared == 0], u[shared == 0])


def test_adaptive_consensus_admm_on_quadratics_converges(oracle):
    """Consensus ADMM on f_k = a_k/2 ||x - b_k||^2 with Eq. 10 applied after
    each consensus (u rescaled) and frozen later still reaches sum a b / sum a
    (Boyd et al., varying penalty)."""
    O = oracle
    rng = np.random.default_rng(6)
    K, P = 3, 14
    a = rng.uniform(0.5, 3.0, (K, 1))
    b = rng.standard_normal((K, P))
    x = np.zeros((K, P)); u = np.zeros((K, P)); z = np.zeros((1, P))
    off = np.array([0, K], np.int64); cp = np.arange(K, dtype=np.int32)
    rho = [50.0] * 5                 # deliberately poor start
    grp = [0] * 3 + [1] * 4 + [2] * 3 + [3] * 3 + [4]
    for t in range(400):
        rv = np.array([rho[g] for g in grp])
        x[:] = (a * b + rv * (z - u)) / (a + rv)
        res = O.consensus(x, u, z, off, cp, 0, alpha=1.0, rho=rho)
        new = O.adaptive_rho(rho, res, t, freeze_after=100)
        O.scale_duals(u, np.ones(K, np.uint8), [o / n for o, n in zip(rho, new)], 0)
        rho = new
    np.testing.assert_allclose(z[0], (a * b).sum(0) / a.sum(), atol=1e-9)
