"""CPU reference of the learned warm start (FP64): features, 3D conv network,
loss, gradients and the interior start point built from a prediction.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no warm start; this module restates, in plain numpy, what the
library's warm-start kernels compute, so their forward and backward passes can
be checked element by element.  The network is four 3x3x3 convolutions with
"same" zero padding over the grid of half-spectrum slots (axes: halved axis,
then the in-plane axes), channels last:

    h1 = relu(conv(x, W1) + b1)      8 -> 32 channels
    h2 = relu(conv(h1, W2) + b2)    32 -> 32
    h3 = relu(conv(h2, W3) + b3)    32 -> 32
    y  = conv(h3, W4) + b4           32 -> 4

conv(x, W)[v, o] = sum_{t in {-1,0,1}^3} sum_i x[v + t, i] W[t + 1, i, o]
(zero outside the grid).  Input features of slot s with beta coordinates
(c_0, c_1) = M_perp^T b at s, scaled by 1/lambda:
    [c_0, c_1, soft(c_0, 1), soft(c_1, 1), |(c_0, c_1)|, kl/(Hl-1), f0, f1]
with f_i = min(k_i, N_i - k_i) / (N_i / 2) (0 for a missing axis).  Outputs:
y[..., 0:2] correct the soft-threshold guess, beta0 = lambda (soft(c) + y[0:2]);
y[..., 2:4] are logits of "coordinate is non-zero".

The start point the IPM is given (``start_point``): with mu0 = mu_scale lambda^2 and
p = sigmoid(logit) per coordinate,
    beta0 = lambda (soft(c / lambda, 1) + y_corr),  z0 = |beta0| + (mu0 / lambda)(2 - p),
    s1 = z0 + beta0,  s2 = z0 - beta0,  nu_i = mu0 / s_i,
so every complementarity product s_i nu_i equals mu0 (the point lies on the
central path's complementarity target for mu0), z0 > |beta0| keeps both slacks
positive, and the rows z - beta - s2 = 0, z + beta - s1 = 0 of Eq. (slackproblem)
hold exactly.  A coordinate predicted inactive (p = 0) gets the slack 2 mu0/lambda
on both sides and nu1 = nu2 = lambda/2 (so nu1 + nu2 = lambda, the row-2 residual
of Eq. (kkt) is 0 there); one predicted active (p = 1) gets mu0/lambda on the side
of its sign.
"""

import numpy as np

TAPS = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]


def conv3d(x, W, b=None):
    """x: (D0, D1, D2, Ci), W: (3, 3, 3, Ci, Co) -> (D0, D1, D2, Co), zero padding."""
    D0, D1, D2, Ci = x.shape
    Co = W.shape[-1]
    xp = np.zeros((D0 + 2, D1 + 2, D2 + 2, Ci))
    xp[1:-1, 1:-1, 1:-1] = x
    y = np.zeros((D0, D1, D2, Co))
    for (a, b_, c) in TAPS:
        y += xp[1 + a:1 + a + D0, 1 + b_:1 + b_ + D1, 1 + c:1 + c + D2] @ W[a + 1, b_ + 1, c + 1]
    if b is not None:
        y += b
    return y


def conv3d_backward(x, W, dy):
    """Gradients of sum(dy * conv3d(x, W)) w.r.t. x, W and the bias."""
    D0, D1, D2, Ci = x.shape
    dyp = np.zeros((D0 + 2, D1 + 2, D2 + 2, dy.shape[-1]))
    dyp[1:-1, 1:-1, 1:-1] = dy
    xp = np.zeros((D0 + 2, D1 + 2, D2 + 2, Ci))
    xp[1:-1, 1:-1, 1:-1] = x
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for (a, b_, c) in TAPS:
        # y[v] gets x[v + t] W[t]  =>  dx[u] += dy[u - t] W[t]^T,  dW[t] += x[v + t]^T dy[v]
        dx += dyp[1 - a:1 - a + D0, 1 - b_:1 - b_ + D1, 1 - c:1 - c + D2] @ W[a + 1, b_ + 1, c + 1].T
        xs = xp[1 + a:1 + a + D0, 1 + b_:1 + b_ + D1, 1 + c:1 + c + D2].reshape(-1, Ci)
        dW[a + 1, b_ + 1, c + 1] = xs.T @ dy.reshape(-1, dy.shape[-1])
    db = dy.reshape(-1, dy.shape[-1]).sum(axis=0)
    return dx, dW, db


def forward(x, params):
    """params: list of (W, b) for the four layers; returns (y, activations)."""
    acts = [x]
    h = x
    for li, (W, b) in enumerate(params):
        z = conv3d(h, W, b)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    return h, acts


def backward(acts, params, dy):
    """Gradients of the loss w.r.t. every (W, b) given dL/dy of the last layer."""
    grads = [None] * len(params)
    g = dy
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li < len(params) - 1:
            g = g * (acts[li + 1] > 0)           # relu'
        dx, dW, db = conv3d_backward(acts[li], W, g)
        grads[li] = (dW, db)
        g = dx
    return grads


def loss_and_grad(y, target, support, w_support=0.1):
    """Mean squared error of y[...,0:2] against target plus w_support times the
    mean binary cross-entropy of the logits y[...,2:4] against support (0/1);
    valid is the mask of LASSO coordinates (ghosts excluded), per output pair."""
    valid = support >= 0
    n = max(1, int(valid.sum()))
    d = np.where(valid, y[..., 0:2] - target, 0.0)
    mse = (d * d).sum() / n
    lg = y[..., 2:4]
    p = 1.0 / (1.0 + np.exp(-lg))
    s = np.where(valid, support, 0.0)
    bce = np.where(valid, np.logaddexp(0.0, lg) - s * lg, 0.0).sum() / n
    dy = np.zeros_like(y)
    dy[..., 0:2] = 2.0 * d / n
    dy[..., 2:4] = np.where(valid, w_support * (p - s) / n, 0.0)
    return mse + w_support * bce, dy


def soft1(u):
    return np.sign(u) * np.maximum(np.abs(u) - 1.0, 0.0)


def slot_grid(dims):
    """Grid of half-spectrum slots the network runs on: (Hl, N0, N1) for 3D,
    (Hl, 1, N0) for 2D, (Hl, 1, 1) for 1D, Hl = N_last/2 + 1."""
    dims = tuple(dims)
    Hl = dims[-1] // 2 + 1
    if len(dims) == 3:
        return (Hl, dims[0], dims[1])
    if len(dims) == 2:
        return (Hl, 1, dims[0])
    return (Hl, 1, 1)


def features(c_slots, lam, dims):
    """Input features (..., 8) from c in slot order, shaped (D0, D1, D2, 2)."""
    D0, D1, D2 = slot_grid(dims)
    c = np.asarray(c_slots, dtype=np.float64).reshape(D0, D1, D2, 2) / lam
    kl = np.arange(D0)[:, None, None] * np.ones((D0, D1, D2))
    k1 = np.arange(D1)[None, :, None] * np.ones((D0, D1, D2))
    k2 = np.arange(D2)[None, None, :] * np.ones((D0, D1, D2))
    f0 = np.minimum(k1, D1 - k1) / (0.5 * D1) if len(dims) == 3 else np.zeros((D0, D1, D2))
    f1 = np.minimum(k2, D2 - k2) / (0.5 * D2) if len(dims) >= 2 else np.zeros((D0, D1, D2))
    x = np.zeros((D0, D1, D2, 8))
    x[..., 0:2] = c
    x[..., 2:4] = soft1(c)
    x[..., 4] = np.sqrt((c * c).sum(-1))
    x[..., 5] = kl / (D0 - 1) if D0 > 1 else 0.0
    x[..., 6] = f0
    x[..., 7] = f1
    return x


def targets(c_slots, bstar_slots, lam, dims, ghost):
    """target (..., 2) = beta*/lambda - soft(c/lambda) and support (..., 2) in {0, 1},
    -1 on ghost coordinates."""
    D0, D1, D2 = slot_grid(dims)
    c = np.asarray(c_slots).reshape(D0, D1, D2, 2) / lam
    b = np.asarray(bstar_slots).reshape(D0, D1, D2, 2)
    t = b / lam - soft1(c)
    sup = (np.abs(b) > 1e-6 * lam).astype(float)
    sup[np.asarray(ghost).reshape(D0, D1, D2, 2)] = -1.0
    return t, sup


def start_point(c, y_corr, logit, lam, mu_scale):
    """Interior start point (beta, z, s1, s2, nu1, nu2) from a prediction, coordinate by
    coordinate (any shape; ghosts are the caller's business): c = M_perp^T b, y_corr the
    network's correction of the soft-threshold guess and logit its support logit."""
    c, y_corr, logit = (np.asarray(a, dtype=np.float64) for a in (c, y_corr, logit))
    mu0 = mu_scale * lam * lam
    beta = lam * (soft1(c / lam) + y_corr)
    p = 1.0 / (1.0 + np.exp(-logit))
    z = np.abs(beta) + (mu0 / lam) * (2.0 - p)
    s1, s2 = z + beta, z - beta
    return beta, z, s1, s2, mu0 / s1, mu0 / s2
