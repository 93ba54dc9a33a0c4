"""The FP64 reference network's backpropagation against central finite
differences (it then judges the GPU network's gradients)."""
import numpy as np

from oracle import oracle as O


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(21)
    npar = O.mlp_nparams()
    assert npar == 2 * 64 + 64 + 2 * (64 * 64 + 64) + 2 * 64 + 2
    P = rng.normal(0.0, 0.3, npar)
    x = rng.uniform(-1, 1, (17, 2))
    t = rng.uniform(-1, 1, (17, 2))
    loss, G = O.mlp_loss_grad(P, x, t)
    idx = np.concatenate([rng.choice(npar, 60, replace=False), [0, 129, npar - 1, npar - 3]])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (O.mlp_loss_grad(Pp, x, t)[0] - O.mlp_loss_grad(Pm, x, t)[0]) / (2 * h)
        assert abs(fd - G[i]) <= 1e-6 * max(1.0, abs(G[i])), (i, fd, G[i])
    # the loss is the mean squared error of the forward pass
    y = O.mlp_forward(P, x)
    assert abs(loss - np.mean(np.sum((y - t) ** 2, axis=1))) < 1e-12
