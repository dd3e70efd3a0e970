"""GPU parity of the stacked-rules + readout + MSE training step (both forms) against the FP64
oracle, plus a central finite-difference check (h = 1e-3) of the GPU gradients in the FP32 form."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import programs, relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import rel_frob

pytestmark = pytest.mark.gpu


def _case(n_tuples=20_000, n_keys=2000, seed=0):
    r1, W2, b2, groups, targets = W.config3(seed=seed, n_tuples=n_tuples, n_keys=n_keys)
    br = r1.branches[0]
    # G(k, g): one group per H key (aligned with h_ids); T(g; z_t) for g = 0..7
    return dict(h=r1.h_ids, z=r1.z, src=br.src, dst=br.dst, W1=br.W, b1=br.b, W2=W2, b2=b2,
                g_keys=r1.h_ids.copy(), g_groups=groups, t_keys=np.arange(8, dtype=np.int32), targets=targets)


def _dev(c, bf16):
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in c.items()}
    return t


def _oracle(c):
    args = (c["h"], c["z"], c["src"], c["dst"], c["W1"], c["b1"], c["W2"], c["b2"], c["g_keys"], c["g_groups"],
            c["t_keys"], c["targets"])
    f = O.stacked_forward(*args)
    g = O.stacked_backward(*args, fwd=f)
    return f, g


def _program(c, bf16):
    t = _dev(c, bf16)
    prog = programs.StackedReadout(t["h"], t["src"], t["dst"], t["g_keys"], t["g_groups"], t["t_keys"],
                                   t["targets"], 64, bf16=bf16)
    return prog, t


@pytest.mark.parametrize("bf16", [False, True])
def test_stacked_step_matches_oracle(gpu, bf16):
    c = _case()
    prog, t = _program(c, bf16)
    loss, grads = prog.step(t["z"], t["W1"], t["b1"], t["W2"], t["b2"])
    torch.cuda.synchronize()
    for p in (prog.p1, prog.p2, prog.p3):
        p.check()
    f, g = _oracle(c)
    assert np.array_equal(prog.k1.cpu().numpy(), f["k1"])
    assert np.array_equal(prog.k2.cpu().numpy(), f["k2"])
    assert np.array_equal(prog.ko.cpu().numpy(), f["ko"])
    tol = 2e-2 if bf16 else 1e-5
    assert abs(float(loss.item()) - f["loss"]) <= tol * abs(f["loss"])
    for name, ref in (("dW1", g["dW1"]), ("db1", g["db1"]), ("dW2", g["dW2"]), ("db2", g["db2"]), ("dz", g["dz"])):
        err = rel_frob(grads[name].cpu().numpy(), ref)
        assert err <= (5e-2 if bf16 else 1e-4), (name, err)


def test_stacked_gradient_finite_differences_fp32(gpu):
    """(L(p + h) - L(p - h)) / 2h on the GPU, h = 1e-3, against the GPU's analytic gradient."""
    c = _case(n_tuples=6000, n_keys=800, seed=1)
    prog, t = _program(c, False)
    loss, grads = prog.step(t["z"], t["W1"], t["b1"], t["W2"], t["b2"])
    L0 = float(loss.item())
    h = 1e-3
    rng = np.random.default_rng(3)
    checked = 0
    for name, gname in (("W1", "dW1"), ("b1", "db1"), ("W2", "dW2"), ("b2", "db2"), ("z", "dz")):
        ten = t[name]
        gr = grads[gname].cpu().numpy()
        flat = np.argsort(-np.abs(gr).reshape(-1))[:20]  # the largest-gradient coordinates
        for fi in rng.choice(flat, size=3, replace=False):
            idx = np.unravel_index(int(fi), ten.shape)
            old = ten[idx].item()
            ten[idx] = old + h
            lp = float(prog.forward(t["z"], t["W1"], t["b1"], t["W2"], t["b2"])[0].item())
            ten[idx] = old - h
            lm = float(prog.forward(t["z"], t["W1"], t["b1"], t["W2"], t["b2"])[0].item())
            ten[idx] = old
            fd = (lp - lm) / (2 * h)
            an = float(gr[idx])
            assert abs(fd - an) <= 5e-2 * abs(an) + 2e-4 * abs(L0) / h * 1e-3 + 1e-6, (name, idx, fd, an)
            checked += 1
    assert checked == 15
