"""Pins of the oracle's learned-far-field pieces (network, loss, AdamW,
pair features, channel sums) against facts that do not come from them:
finite differences of the forward pass, the closed form of GELU at known
points and of a network with zeroed layers, the closed form of the first
Adam step, rotation/translation invariance of the features, and the
monopole of a one-member cluster being exact."""

import math

import numpy as np
import pytest

from paper_2509_22110_gb300 import meshgen


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod


def rand_params(rng, n, scale=0.3):
    return rng.standard_normal(n) * scale


def test_backward_matches_finite_differences(orc):
    rng = np.random.default_rng(0)
    n = orc.mlp_nparam()
    P = rand_params(rng, n)
    X = rng.standard_normal((5, 24))
    T = rng.standard_normal((5, 7))
    M = (rng.uniform(size=(5, 7)) > 0.3).astype(np.float64)
    L, g = orc.mlp_loss_grad(P, X, T, M)
    idx = rng.choice(n, 60, replace=False)
    h = 1e-4

    def loss_at(i, t):
        Q = P.copy()
        Q[i] += t
        return orc.mlp_loss_grad(Q, X, T, M)[0]

    for i in idx:
        # fourth-order central difference
        fd = (-loss_at(i, 2 * h) + 8 * loss_at(i, h) - 8 * loss_at(i, -h) + loss_at(i, -2 * h)) / (12 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1e-3, abs(g[i])) + 1e-11, (i, fd, g[i])


def test_gelu_closed_form_through_the_network(orc):
    """W1..W3 = 0 makes every hidden unit g(b); with b3 = 1 and one output
    reading one unit, y = g(1) = (1 + tanh(sqrt(2/pi) 1.044715)) / 2."""
    n = orc.mlp_nparam()
    P = np.zeros(n)
    off_b3 = 64 * 24 + 64 + 64 * 64 + 64 + 64 * 64
    off_w4 = off_b3 + 64
    P[off_b3:off_b3 + 64] = 1.0
    P[off_w4 + 0 * 64 + 5] = 1.0  # output 0 reads hidden unit 5
    P[off_w4 + 3 * 64 + 7] = -2.0  # output 3 = -2 g(1)
    off_b4 = off_w4 + 7 * 64
    P[off_b4 + 6] = 0.25
    y = orc.mlp_forward(P, np.random.default_rng(1).standard_normal((3, 24)))
    phi1 = 0.5 * (1 + math.tanh(math.sqrt(2 / math.pi) * 1.044715))
    assert abs(phi1 - 0.8411919906082768) < 1e-15
    np.testing.assert_allclose(y[:, 0], phi1, rtol=1e-15)
    np.testing.assert_allclose(y[:, 3], -2 * phi1, rtol=1e-15)
    np.testing.assert_allclose(y[:, 6], 0.25, rtol=1e-15)
    np.testing.assert_allclose(y[:, [1, 2, 4, 5]], 0.0, atol=1e-15)


def test_gelu_negative_tail(orc):
    """g(-b) -> 0 for large b: a network whose last hidden layer sits at -8 outputs b4."""
    n = orc.mlp_nparam()
    P = np.zeros(n)
    off_b3 = 64 * 24 + 64 + 64 * 64 + 64 + 64 * 64
    P[off_b3:off_b3 + 64] = -8.0
    off_w4 = off_b3 + 64
    P[off_w4:off_w4 + 7 * 64] = 1.0
    y = orc.mlp_forward(P, np.zeros((1, 24)))
    assert np.all(np.abs(y) < 64 * 8 * 1e-14)


def test_adamw_first_step_closed_form(orc):
    """At t = 1 the bias-corrected moments are g and g^2, so
    w1 = w0 - lr g / (|g| + eps) - lr wd w0."""
    rng = np.random.default_rng(2)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    w0 = w.copy()
    m = np.zeros(50)
    v = np.zeros(50)
    lr, wd, eps = 1e-3, 1e-2, 1e-8
    orc.adamw_step(w, m, v, g, lr, 0.9, 0.999, eps, wd, 1)
    np.testing.assert_allclose(w, w0 - lr * g / (np.abs(g) + eps) - lr * wd * w0, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_features_rotation_translation_invariant(orc):
    V, F = meshgen.sh_deformed_sphere(3, 12, 0.05, 2)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    for VV in (V, V @ Q.T + np.array([3.0, -1.0, 0.5])):
        x, nu, w = orc.tri_data(VV, F)
        # two fixed groups of triangles, moments summed directly (independent of the tree)
        gL = np.arange(0, 12)
        gC = np.arange(600, 700)

        def mom_of(g):
            A = w[g].sum()
            nn = nu[g]
            m2 = [(w[g] * nn[:, a] * nn[:, b]).sum() for a, b in [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]]
            return np.array([A, *(w[g, None] * x[g]).sum(0), *(w[g, None] * nn).sum(0), *m2])

        def box_of(g):
            vv = VV[F[g].ravel()]
            return np.concatenate([vv.min(0), vv.max(0)])

        f = orc.far_features(mom_of(gL), box_of(gL), mom_of(gC), box_of(gC))
        if VV is V:
            f0 = f
    # boxes are axis aligned, so the two diagonal features change under rotation; the rest must not
    keep = [i for i in range(24) if i not in (2, 3)]
    np.testing.assert_allclose(f[keep], f0[keep], rtol=1e-10, atol=1e-12)


def test_single_member_cluster_monopole_is_exact(orc):
    """A cluster of one triangle has X = x_S, nubar = nu_S, A = w_S: the
    monopole equals the member sum in every channel."""
    V, F = meshgen.sh_deformed_sphere(3, 12, 0.05, 2)
    x, nu, w = orc.tri_data(V, F)
    S = 700
    momC = np.array([w[S], *(w[S] * x[S]), *(w[S] * nu[S]), *[w[S] * nu[S, a] * nu[S, b] for a, b in
                                                              [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]]])
    mono, exact = orc.far_channels(x, nu, w, np.arange(0, 9), [S], momC)
    np.testing.assert_allclose(exact, mono, rtol=1e-12)
    assert np.all(mono[[0, 1]] > 0)


def test_channel_energy_matches_pair_sums(orc):
    """Channels 0 and 1 summed over a group pair are lambda times the sums of
    e_TS and e_ST over that group pair, written out independently here."""
    V, F = meshgen.sh_deformed_sphere(3, 12, 0.05, 2)
    x, nu, w = orc.tri_data(V, F)
    tl = np.arange(0, 10)
    sc = np.arange(500, 560)
    A = w[sc].sum()
    momC = np.array([A, *(w[sc, None] * x[sc]).sum(0), *(w[sc, None] * nu[sc]).sum(0), 0, 0, 0, 0, 0, 0])
    _, exact = orc.far_channels(x, nu, w, tl, sc, momC)
    eTS = eST = 0.0
    for T in tl:
        for S in sc:
            d = x[T] - x[S]
            r2 = d @ d
            eTS += w[T] * w[S] * (nu[T] @ d) ** 6 / r2**6
            eST += w[T] * w[S] * (nu[S] @ -d) ** 6 / r2**6
    np.testing.assert_allclose(exact[0], 2 * eTS, rtol=1e-12)
    np.testing.assert_allclose(exact[1], 2 * eST, rtol=1e-12)
