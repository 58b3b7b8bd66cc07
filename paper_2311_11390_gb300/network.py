"""Classification network on the library kernels (the network of the classification
experiments, Section 4.2 and Supplementary "Classification"):

    input spike raster -> projection (tcgen05, split-BF16) -> ALIF layer
                       -> projection -> ALIF layer
                       -> leaky readout (integrator without spike or reset, summed over time)
                       -> softmax cross-entropy.

Each stage is a torch.autograd.Function over the C ABI.  Spikes travel between layers as
float 0/1 tensors (the autograd handle, receiving dL/dS) together with their bit words
(what the next projection and the readout consume).  The input raster enters as bits only.
"""
from __future__ import annotations

import numpy as np
import torch

from . import alif
from .autograd import ALIFFunction


class SynProject(torch.autograd.Function):
    """I = W S + bias from spike words [B, Nin, ceil(T/32)]; S (float, optional) is the
    autograd handle of the same spikes and receives dL/dS = W^T dL/dI."""

    @staticmethod
    def forward(ctx, S, W, bias, words, T):
        Wd = W.detach().contiguous()
        hi, lo = alif.split_bf16(Wd)
        I = alif.syn_project(words, hi, lo, None if bias is None else bias.detach().contiguous(),
                             Nin=W.shape[1], T=T)
        ctx.save_for_backward(Wd)
        ctx.words = words
        ctx.has_S = S is not None
        ctx.has_bias = bias is not None
        return I

    @staticmethod
    def backward(ctx, gI):
        (W,) = ctx.saved_tensors
        need_S = ctx.has_S and ctx.needs_input_grad[0]
        need_b = ctx.has_bias and ctx.needs_input_grad[2]
        gW, gS, gb = alif.syn_project_backward(ctx.words, gI.contiguous(), W=W, Nin=W.shape[1],
                                               want_gW=ctx.needs_input_grad[1], want_gS=need_S, want_gb=need_b)
        return gS, gW, gb, None, None


class Readout(torch.autograd.Function):
    """Leaky readout summed over time: logits [B, C] from the last layer's spikes."""

    @staticmethod
    def forward(ctx, S, W, bias, words, T, w_t, w_sum):
        logits, counts = alif.readout_forward(words, T, W.detach().contiguous(),
                                              None if bias is None else bias.detach().contiguous(), w_t, w_sum)
        ctx.save_for_backward(W.detach().contiguous(), counts, w_t)
        ctx.T, ctx.w_sum, ctx.has_bias = T, w_sum, bias is not None
        return logits

    @staticmethod
    def backward(ctx, g):
        W, counts, w_t = ctx.saved_tensors
        gS, gW, gb = alif.readout_backward(W, w_t, ctx.w_sum, counts, g.contiguous(), ctx.T,
                                           want_spikes=ctx.needs_input_grad[0], want_W=ctx.needs_input_grad[1],
                                           want_bias=ctx.has_bias and ctx.needs_input_grad[2])
        return gS, gW, gb, None, None, None, None


class CrossEntropy(torch.autograd.Function):
    """Mean softmax cross-entropy of logits [B, C] against int32 labels [B]."""

    @staticmethod
    def forward(ctx, logits, labels):
        loss, g = alif.cross_entropy(logits.detach().contiguous(), labels, want_grad=True)
        ctx.save_for_backward(g)
        return loss[0]

    @staticmethod
    def backward(ctx, go):
        (g,) = ctx.saved_tensors
        return g * go, None


class ALIFNet(torch.nn.Module):
    """Nin -> H1 -> H2 ALIF layers -> C-class leaky readout.  Initialisation of the paper's
    classification runs: weights U(+-1/sqrt(fan_in)), tau_mem 20 ms, tau_adapt 150 ms,
    d 1.8, threshold baseline 1; hidden biases are given (the synthetic inputs need them to
    drive the layers)."""

    def __init__(self, n_in, hidden=(256, 256), n_classes=20, dt=1.0, arp=2.0, tau_out=20.0, slope=25.0,
                 hidden_bias=(0.8, 1.6), seed=0, device="cuda"):
        super().__init__()
        g = np.random.default_rng(seed)
        dims = [n_in, *hidden]
        self.W = torch.nn.ParameterList()
        self.b = torch.nn.ParameterList()
        self.tau_mem = torch.nn.ParameterList()
        self.tau_adapt = torch.nn.ParameterList()
        self.theta0 = torch.nn.ParameterList()
        self.d = torch.nn.ParameterList()
        P = lambda a: torch.nn.Parameter(torch.from_numpy(np.asarray(a, np.float32)).to(device))
        for fi, fo in zip(dims[:-1], dims[1:]):
            lim = 1.0 / np.sqrt(fi)
            self.W.append(P(g.uniform(-lim, lim, (fo, fi))))
            self.b.append(P(g.uniform(*hidden_bias, fo)))
            self.tau_mem.append(P(np.full(fo, 20.0)))
            self.tau_adapt.append(P(np.full(fo, 150.0)))
            self.theta0.append(P(np.full(fo, 1.0)))
            self.d.append(P(np.full(fo, 1.8)))
        lim = 1.0 / np.sqrt(dims[-1])
        self.W_out = P(g.uniform(-lim, lim, (n_classes, dims[-1])))
        self.b_out = P(np.zeros(n_classes))
        self.dt, self.arp, self.tau_out, self.slope = dt, arp, tau_out, slope
        self._w = {}

    @classmethod
    def from_workload(cls, w, slope=25.0, device="cuda"):
        """Network with the weights, biases and neuron parameters of a synth.classification
        workload (hidden sizes and class count taken from it)."""
        hidden = tuple(b.shape[0] for b in w.bias)
        net = cls(w.W[0].shape[1], hidden, w.W[-1].shape[0], dt=w.dt, arp=w.arp, tau_out=w.tau_out,
                  slope=slope, device=device)
        with torch.no_grad():
            for l in range(len(hidden)):
                net.W[l].copy_(torch.from_numpy(w.W[l]))
                net.b[l].copy_(torch.from_numpy(w.bias[l]))
                net.tau_mem[l].copy_(torch.from_numpy(np.asarray(w.params[l].tau_mem, np.float32)))
                net.tau_adapt[l].copy_(torch.from_numpy(np.asarray(w.params[l].tau_adapt, np.float32)))
                net.theta0[l].copy_(torch.from_numpy(np.asarray(w.params[l].theta0, np.float32)))
                net.d[l].copy_(torch.from_numpy(np.asarray(w.params[l].d, np.float32)))
            net.W_out.copy_(torch.from_numpy(w.W[-1]))
        return net

    def readout_weights(self, T, device):
        key = (T, str(device))
        if key not in self._w:
            self._w[key] = alif.readout_weights(T, self.dt, self.tau_out, device)
        return self._w[key]

    def forward(self, in_words: torch.Tensor, T: int, keep=None):
        """in_words: int32 [B, Nin, ceil(T/32)] input spike bits -> logits [B, C].
        keep: optional dict that receives the intermediate tensors (I, S, words per layer)."""
        S, words = None, in_words
        for l in range(len(self.W)):
            I = SynProject.apply(S, self.W[l], self.b[l], words, T)
            S, words = ALIFFunction.apply(I, self.tau_mem[l], self.tau_adapt[l], self.theta0[l], self.d[l], None,
                                          self.dt, self.arp, self.slope)
            if keep is not None:
                keep[f"I{l}"], keep[f"S{l}"], keep[f"words{l}"] = I, S, words
        w_t, w_sum = self.readout_weights(T, in_words.device)
        return Readout.apply(S, self.W_out, self.b_out, words, T, w_t, w_sum)

    def loss(self, in_words, labels, T, keep=None):
        logits = self.forward(in_words, T, keep)
        if keep is not None:
            keep["logits"] = logits
        return CrossEntropy.apply(logits, labels)
