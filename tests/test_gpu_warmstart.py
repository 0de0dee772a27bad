"""Learned warm start: BF16 tensor-core kernels against the FP64 CPU reference,
and what the trained network gains over the cold start (needs a GPU).

Tolerances: conv inputs are BF16-exact, so the kernels differ from the FP64
reference only by FP32 accumulation over at most 27 x 32 = 864 products
(relative ~1e-6; we allow 1e-4 of the output scale).  The whole-network
gradient also rounds every activation and gradient to BF16 (8-bit mantissa,
relative 2^-9 per rounding, four layers): we require relative norm error below
5 % and cosine similarity above 0.995 against the FP64 reference fed the same
BF16-rounded weights.
"""

import numpy as np
import pytest
import torch

from oracle import warmstart as ows
from oracle.lasso import Problem
from paper_2502_04217_gb300 import binding
from paper_2502_04217_gb300.synth import make_problem

from layout import ghost_mask, oracle_to_lib

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)


def dev_bf16(a):
    return bf16(a).cuda().contiguous()


def as_u16(t):
    return t.view(torch.int16)


# D2 >= 64 runs the tcgen05 kernel (128-voxel tiles along D2, segments of 32
# steps along D1: ragged tiles, several segments, zero padding on every face);
# smaller D2 the mma.sync kernel.
@pytest.mark.parametrize("cin,cout,dims", [(32, 32, (3, 5, 70)), (16, 32, (2, 3, 13)), (32, 8, (4, 2, 64)),
                                           (16, 8, (1, 1, 5)), (32, 32, (2, 2, 129)), (32, 32, (3, 40, 256)),
                                           (16, 32, (2, 33, 128)), (32, 8, (3, 4, 200)), (16, 8, (2, 2, 64)),
                                           (32, 32, (1, 1, 384))])
def test_conv_forward_matches_reference(cin, cout, dims):
    rng = np.random.default_rng(1)
    x = bf16(rng.standard_normal(dims + (cin,)))
    w = bf16(0.2 * rng.standard_normal((27, cout, cin)))
    b = rng.standard_normal(cout).astype(np.float32)
    aux = bf16(rng.standard_normal(dims + (cout,)))
    for relu, use_aux in [(0, False), (1, False), (0, True)]:
        y = torch.empty(int(np.prod(dims)) * cout, dtype=torch.float32, device="cuda")
        binding.ws_conv_forward(cin, cout, dims, as_u16(x.cuda().contiguous()), as_u16(w.cuda().contiguous()),
                                torch.as_tensor(b).cuda(), relu, as_u16(aux.cuda().contiguous()) if use_aux else None, y)
        W = w.float().numpy().reshape(3, 3, 3, cout, cin).transpose(0, 1, 2, 4, 3)
        ref = ows.conv3d(x.float().numpy().astype(np.float64), W.astype(np.float64), b.astype(np.float64))
        if relu:
            ref = np.maximum(ref, 0)
        if use_aux:
            ref = ref * (aux.float().numpy() > 0)
        got = y.cpu().numpy().reshape(dims + (cout,))
        assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


def test_conv_pipeline_wait_expires_with_an_error():
    """Failure detection without a GPU fault: one TMA copy of the tcgen05 pipeline
    never arrives (a barrier nothing completes); every pipeline wait is bounded,
    so the call returns IPM_TIMEOUT instead of hanging, and the next call on the
    same context computes the right result."""
    dims, cin, cout = (3, 40, 256), 32, 32
    rng = np.random.default_rng(3)
    x = bf16(rng.standard_normal(dims + (cin,)))
    w = bf16(0.2 * rng.standard_normal((27, cout, cin)))
    b = rng.standard_normal(cout).astype(np.float32)
    args = (as_u16(x.cuda().contiguous()), as_u16(w.cuda().contiguous()), torch.as_tensor(b).cuda(), 1, None)
    y = torch.empty(int(np.prod(dims)) * cout, dtype=torch.float32, device="cuda")
    binding.ws_test_conv_stall(5, 14)
    with pytest.raises(binding.IpmError) as e:
        binding.ws_conv_forward(cin, cout, dims, *args, y)
    assert e.value.status == binding.IPM_TIMEOUT and "expired" in str(e.value)
    binding.ws_conv_forward(cin, cout, dims, *args, y)
    W = w.float().numpy().reshape(3, 3, 3, cout, cin).transpose(0, 1, 2, 4, 3)
    ref = np.maximum(ows.conv3d(x.float().numpy().astype(np.float64), W.astype(np.float64), b.astype(np.float64)), 0)
    assert np.abs(y.cpu().numpy().reshape(dims + (cout,)) - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())
    with pytest.raises(binding.IpmError):
        binding.ws_test_conv_stall(0, 14)


@pytest.mark.parametrize("cin,m,mout,dims", [(32, 32, 32, (3, 4, 70)), (16, 32, 32, (2, 3, 17)),
                                             (32, 16, 8, (3, 2, 65)), (16, 16, 16, (1, 1, 9))])
def test_conv_weight_gradient_matches_reference(cin, m, mout, dims):
    rng = np.random.default_rng(2)
    x = bf16(rng.standard_normal(dims + (cin,)))
    dy = bf16(rng.standard_normal(dims + (m,)))
    dw = torch.empty(27 * mout * cin, dtype=torch.float32, device="cuda")
    db = torch.empty(mout, dtype=torch.float32, device="cuda")
    binding.ws_conv_wgrad(cin, m, mout, dims, as_u16(x.cuda().contiguous()), as_u16(dy.cuda().contiguous()), dw, db)
    W0 = np.zeros((3, 3, 3, cin, m))
    _, dW, dB = ows.conv3d_backward(x.float().numpy().astype(np.float64), W0, dy.float().numpy().astype(np.float64))
    ref = dW.reshape(27, cin, m).transpose(0, 2, 1)[:, :mout, :]
    got = dw.cpu().numpy().reshape(27, mout, cin)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= 1e-4 * scale
    assert np.abs(db.cpu().numpy() - dB[:mout]).max() <= 1e-4 * max(1.0, np.abs(dB).max())


def _layers(params_flat):
    """Split the FP32 parameter vector into the oracle's (W, b) list, weights rounded to BF16."""
    shapes = [(16, 32, 8, 32), (32, 32, 32, 32), (32, 32, 32, 32), (32, 8, 32, 4)]  # cin, cout, cin_real, cout_real
    out, o = [], 0
    for cin, cout, cir, cor in shapes:
        W = params_flat[o:o + 27 * cout * cin].reshape(27, cout, cin)
        o += 27 * cout * cin
        b = params_flat[o:o + cout]
        o += cout
        Wb = torch.as_tensor(W).to(torch.bfloat16).float().numpy().astype(np.float64)
        out.append((Wb.reshape(3, 3, 3, cout, cin).transpose(0, 1, 2, 4, 3)[:, :, :, :cir, :cor].copy(),
                    b[:cor].astype(np.float64)))
    return out


def test_network_gradient_matches_reference():
    from oracle import ipm as oipm
    dims = (8, 12, 16)
    w = make_problem("custom", dims=dims, missing=0.15, seed=60)
    prob = Problem(dims, w.mask.astype(bool), w.y, 1.0)
    prob.lam = 0.1 * prob.lambda_max()
    # the training target is the oracle's own solution (nothing the reference sees comes from the GPU)
    bstar_o = oipm.solve(prob, gap_tol=1e-8)["beta"]
    opt = binding.default_options(lambda_relative=0)
    h = binding.ipm_create(dims, w.mask, w.y, prob.lam, opt)
    net = binding.ws_create(seed=7)
    try:
        res = {"lambda": prob.lam}
        H, n = binding.ipm_sizes(h)
        bstar = oracle_to_lib(h, bstar_o, dims)
        loss = binding.ws_train_step(net, h, bstar, 0.0)
        npar = binding.ws_num_params(net)
        params = np.empty(npar, dtype=np.float32)
        grads = np.empty(npar, dtype=np.float32)
        binding.ws_get_params(net, params)
        binding.ws_get_grads(net, grads)
        y = torch.empty(H * 8, dtype=torch.float32, device="cuda")
        binding.ws_forward(net, h, y)
        # reference on the same slot grid
        c_lib = oracle_to_lib(h, prob.c, dims).cpu().numpy()
        x = ows.features(c_lib, res["lambda"], dims)
        x = torch.as_tensor(x.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
        layers = _layers(params)
        yr, acts = ows.forward(x, layers)
        t, sup = ows.targets(c_lib, bstar.cpu().numpy(), res["lambda"], dims, ghost_mask(h, dims))
        lref, dy = ows.loss_and_grad(yr, t, sup)
        gref = ows.backward(acts, layers, dy)
        ygot = y.cpu().numpy().reshape(yr.shape[:3] + (8,))[..., :4]
        assert np.linalg.norm(ygot - yr) <= 0.02 * np.linalg.norm(yr)
        assert abs(loss - lref) <= 0.02 * abs(lref)
        got, ref = [], []
        o = 0
        for (cin, cout, cir, cor), (dWr, dbr) in zip([(16, 32, 8, 32), (32, 32, 32, 32), (32, 32, 32, 32), (32, 8, 32, 4)],
                                                     gref):
            G = grads[o:o + 27 * cout * cin].reshape(3, 3, 3, cout, cin).transpose(0, 1, 2, 4, 3)[:, :, :, :cir, :cor]
            o += 27 * cout * cin
            gb = grads[o:o + cout][:cor]
            o += cout
            got += [G.ravel(), gb]
            ref += [dWr.ravel(), dbr]
        got, ref = np.concatenate(got), np.concatenate(ref)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref))
        assert rel < 0.05 and cos > 0.995, (rel, cos)
    finally:
        binding.ws_destroy(net)
        binding.ipm_destroy(h)


def _params(layers):
    """FP32 parameter vector from per-layer (W [27][cout][cin], b [cout]) in the stored channel counts."""
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers]).astype(np.float32)


def _zero_layers():
    return [(np.zeros((27, cout, cin), np.float32), np.zeros(cout, np.float32))
            for cin, cout in [(16, 32), (32, 32), (32, 32), (32, 8)]]


@pytest.mark.parametrize("dims", [(6, 10, 14), (12, 20), (30,), (5, 9, 7)])
def test_features_kernel_matches_oracle(dims):
    """The input features of every slot against the oracle's definition, element by
    element.  The network is set to pass four features straight to its output: the
    centre tap of layer 1 splits each feature x into relu(x) and relu(-x), layers 2 and 3
    copy them (identity centre tap), and layer 4 forms relu(x) - relu(-x) = x.  All
    products are by 1 and sums have one non-zero term, so y is the BF16 feature exactly;
    the oracle's FP64 feature is rounded to BF16 the same way (through FP32)."""
    w = make_problem("custom", dims=dims, missing=0.1, seed=62)
    prob = Problem(dims, w.mask.astype(bool), w.y, 1.0)
    lam = 0.1 * prob.lambda_max()
    h = binding.ipm_create(dims, w.mask, w.y, lam, binding.default_options(lambda_relative=0))
    net = binding.ws_create(seed=9)
    try:
        H, n = binding.ipm_sizes(h)
        c_lib = oracle_to_lib(h, prob.c, dims).cpu().numpy()
        ref = ows.features(c_lib, lam, dims).reshape(-1, 8)
        ref = torch.as_tensor(ref.astype(np.float32)).to(torch.bfloat16).float().numpy()
        got = np.zeros_like(ref)
        for half in (0, 1):
            L = _zero_layers()
            for i in range(8):
                L[0][0][13, i, i] = 1.0
                L[0][0][13, 8 + i, i] = -1.0
            for l in (1, 2):
                for o in range(16):
                    L[l][0][13, o, o] = 1.0
            for j in range(4):
                L[3][0][13, j, 4 * half + j] = 1.0
                L[3][0][13, j, 8 + 4 * half + j] = -1.0
            binding.ws_set_params(net, _params(L))
            y = torch.empty(H * 8, dtype=torch.float32, device="cuda")
            binding.ws_forward(net, h, y)
            got[:, 4 * half:4 * half + 4] = y.cpu().numpy().reshape(H, 8)[:, :4]
        ulp = np.abs(ref) * 2.0 ** -8 + 1e-30
        assert np.all(np.abs(got - ref) <= ulp), np.abs(got - ref).max()
        assert np.mean(got == ref) > 0.99
    finally:
        binding.ws_destroy(net)
        binding.ipm_destroy(h)


@pytest.mark.parametrize("bias", [(0.25, -0.125, 0.0, 0.0), (-1.5, 2.0, 3.0, -2.5), (0.0, 0.0, -8.0, 8.0)])
def test_start_point_kernel_matches_oracle(bias):
    """The interior start point built from a prediction against the oracle's
    start_point, element by element: every weight 0 and the last layer's bias set, so
    the network's outputs are exactly (y0, y1, logit0, logit1) = bias at every slot;
    the point then varies with c = M_perp^T b from slot to slot."""
    dims = (12, 10, 16)
    w = make_problem("custom", dims=dims, missing=0.1, seed=63)
    prob = Problem(dims, w.mask.astype(bool), w.y, 1.0)
    lam = 0.05 * prob.lambda_max()
    h = binding.ipm_create(dims, w.mask, w.y, lam, binding.default_options(lambda_relative=0))
    net = binding.ws_create(seed=10)
    try:
        L = _zero_layers()
        L[3][1][:4] = bias
        binding.ws_set_params(net, _params(L))
        mu_scale = 0.5
        binding.ws_predict(net, h, mu_scale)
        H, n = binding.ipm_sizes(h)
        pt = [torch.empty(2 * H, dtype=torch.float64, device="cuda") for _ in range(6)]
        binding.ipm_get_point(h, pt)
        got = [v.cpu().numpy() for v in pt]
        c_lib = oracle_to_lib(h, prob.c, dims).cpu().numpy()
        cc = np.arange(2 * H) & 1
        y_corr = np.where(cc == 0, bias[0], bias[1])
        logit = np.where(cc == 0, bias[2], bias[3])
        ref = ows.start_point(c_lib, y_corr, logit, lam, mu_scale)
        ghost = ghost_mask(h, dims)
        # beta0 in FP64; the sigmoid in FP32 (relative 1.2e-7) moves the margin
        # delta = (mu0/lambda)(2 - p) of z, s1, s2 by at most 1.2e-7 mu0/lambda, and
        # nu = mu0 / s (s >= mu0/lambda) by at most 1.2e-7 relative
        mu0 = mu_scale * lam * lam
        for k, (g, r) in enumerate(zip(got, ref)):
            assert np.all(g[ghost] == 0.0)
            g, r = g[~ghost], r[~ghost]
            if k == 0:
                tol = 1e-12 * np.maximum(1.0, np.abs(r))
            elif k <= 3:
                tol = 1e-12 * np.maximum(1.0, np.abs(r)) + 2e-7 * mu0 / lam
            else:
                tol = (1e-12 + 2e-7) * np.abs(r)
            assert np.all(np.abs(g - r) <= tol), (k, float(np.max(np.abs(g - r) / tol)))
    finally:
        binding.ws_destroy(net)
        binding.ipm_destroy(h)


def test_training_steps_reduce_the_loss():
    dims = (16, 16, 16)
    w = make_problem("custom", dims=dims, missing=0.1, seed=61)
    opt = binding.default_options(lambda_relative=1, gap_tol=1e-8)
    h = binding.ipm_create(dims, w.mask, w.y, 0.1, opt)
    net = binding.ws_create(seed=8)
    try:
        binding.ipm_solve(h)
        H, n = binding.ipm_sizes(h)
        pt = [torch.empty(2 * H, dtype=torch.float64, device="cuda") for _ in range(6)]
        binding.ipm_get_point(h, pt)
        losses = [binding.ws_train_step(net, h, pt[0], 3e-3) for _ in range(30)]
        assert losses[-1] < 0.5 * losses[0]
    finally:
        binding.ws_destroy(net)
        binding.ipm_destroy(h)


def test_trained_network_beats_the_cold_start():
    """What the learned part gains: a network trained on 24 solved 32^3 instances
    starts held-out solves closer to the solution, so they need fewer IPM
    iterations; the cold-start IPM stays the arbiter: both reach the same gap and
    their objectives agree within it."""
    from paper_2502_04217_gb300 import warmstart as ws
    data = ws.Dataset(32, 24, seed=0, gap_tol=1e-8)
    net = binding.ws_create(seed=1)
    try:
        hist = ws.train(net, data, epochs=15, lr=1e-3)
        assert min(hist[-3:]) < 0.5 * hist[0]
        opt = binding.default_options(precision=binding.IPM_MIXED, lambda_relative=1, gap_tol=1e-6)
        cold, warm = [], []
        for i in range(6):
            w = ws.instance(32, 1000 + i)
            h = binding.ipm_create(w.dims, w.mask, w.y, w.lam_rel, opt)
            try:
                rc = binding.ipm_solve(h)
                binding.ws_predict(net, h, 0.1)
                rw = binding.ipm_solve(h)
            finally:
                binding.ipm_destroy(h)
            assert rc["rel_gap"] <= 1e-6 and rw["rel_gap"] <= 1e-6
            assert abs(rw["primal"] - rc["primal"]) <= 2e-6 * abs(rc["primal"])
            cold.append(rc["ipm_iters"])
            warm.append(rw["ipm_iters"])
        assert np.mean(warm) <= np.mean(cold) - 1.5, (cold, warm)
    finally:
        binding.ws_destroy(net)
        data.close()
