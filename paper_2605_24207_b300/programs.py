"""Rule programs composed from library calls (no arithmetic here: every step runs in librelnn).

StackedReadout is the training configuration of two stacked join rules, a SUM readout and an MSE
loss relation (a program of the kind of the paper's Sec. 3.6 example):

    H1(d; SUM ReLU(Linear1(Concat(z_s, z_d)))) :- E(s, d), H(s; z_s), H(d; z_d)
    H2(d; SUM Linear2(Concat(z_s, z_d)))       :- E(s, d), H1(s; z_s), H1(d; z_d)
    Out(g; SUM z)                              :- H2(k; z), G(k, g)
    L(; mean((z_o - z_t)^2))                   :- Out(g; z_o), T(g; z_t)

The content track of each rule is planned once (relnn_rule_plan) and reused by every forward and
backward, as the paper caches content across training iterations; an f32 embedding table is
converted to bf16 once per tensor version (relnn_plan_set_z_version), not once per call.
"""
from __future__ import annotations

import torch

from . import relnn as R


class StackedReadout:
    def __init__(self, h_ids, src, dst, g_keys, g_groups, t_keys, targets, d: int, bf16: bool = True,
                 kahan: bool = True, stream=None):
        self.d, self.bf16 = d, bf16
        self.t_keys, self.targets = t_keys, targets
        f = (R.FLAG_BF16 | R.FLAG_RELU_MASK) if bf16 else 0
        if kahan:
            f |= R.FLAG_KAHAN
        self.p1 = R.RulePlan(h_ids, [(src, dst)], d, d, act=R.ACT_RELU, flags=f, stream=stream)
        self.k1 = self.p1.out_keys(stream)
        self.p2 = R.RulePlan(self.k1, [(src, dst)], d, d, act=R.ACT_NONE, flags=f & ~R.FLAG_RELU_MASK,
                             stream=stream)
        self.k2 = self.p2.out_keys(stream)
        ro = R.FLAG_IDENTITY | R.FLAG_NO_JOIN_DST | (R.FLAG_KAHAN if kahan else 0)
        self.p3 = R.RulePlan(self.k2, [(g_keys, g_groups)], d, 0, flags=ro, stream=stream)
        self.ko = self.p3.out_keys(stream)
        self.tuples = self.p1.n_matched + self.p2.n_matched  # rule tuples per step (readout excluded)

    def forward(self, z, W1, b1, W2, b2, stream=None):
        """Loss (device f32 [1]) and the intermediate relations (kept for backward)."""
        h1 = self.p1.forward(z, [W1], [b1], stream=stream, z_version="auto")
        h2 = self.p2.forward(h1, [W2], [b2], stream=stream, z_version="auto")
        ho = self.p3.forward(h2, stream=stream)
        loss, d_ho = R.mse_loss(ho, self.ko, self.targets, self.t_keys, stream=stream)
        self._saved = (z, W1, b1, W2, b2, h1, h2, d_ho)
        return loss, (h1, h2, ho)

    def backward(self, stream=None):
        """Gradients of the last forward's loss: dict with dW1, db1, dW2, db2, dz."""
        z, W1, b1, W2, b2, h1, h2, d_ho = self._saved
        _, _, d_h2, _ = self.p3.backward(d_ho, h2, stream=stream)
        (dW2,), (db2,), d_h1, _ = self.p2.backward(d_h2, h1, [W2], [b2], stream=stream, z_version="auto")
        (dW1,), (db1,), dz, _ = self.p1.backward(d_h1, z, [W1], [b1], stream=stream, z_version="auto")
        return dict(dW1=dW1, db1=db1, dW2=dW2, db2=db2, dz=dz)

    def step(self, z, W1, b1, W2, b2, stream=None):
        """One training step (forward + backward); returns (loss tensor, grads)."""
        loss, _ = self.forward(z, W1, b1, W2, b2, stream=stream)
        return loss, self.backward(stream=stream)
