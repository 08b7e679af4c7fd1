"""Allegro-shaped energy model in FP64 on the CPU (oracle).

The paper (Sec. 2.1) fixes: E = sum of pairwise embedding energies E_ij over
pairs inside a finite cutoff, E(3)-equivariant through tensors up to rank l
and their irreducible tensor products; forces are f_i = -dE/dr_i (Eq. 1).
Everything below that is not in the paper is a stated reading:

  per ordered pair (i, j, n), Delta = r_j + n L - r_i, d = |Delta|, u = Delta/d
    B_k(d)  = sqrt(2/rc) sin(k pi d / rc) / d,          k = 1 .. Nb
    fc(d)   = 1 - 28 x^6 + 48 x^7 - 21 x^8, x = d/rc     (p = 6 envelope)
    Y_l(u)  = real spherical harmonics (oracle.sph)
  two-body latent: x0 = fc * MLP_2b([onehot Z_i, onehot Z_j, B])
  initial tensors: w0 = Lin(x0) (C (lmax+1) values, index c*(lmax+1)+l),
                   V0[c, l m] = w0[c, l] Y_lm
  layer k = 1 .. L:
    e     = Lin_env(x^{k-1})                                  (C values)
    G_i   = (1/sqrt(nu)) sum_{pairs (i, j)} e_ij[c] Y_ij[l m]   (per atom i)
    T[c, path, m3] = sum C^{l1 l2 l3}[m1, m2, m3] V^{k-1}_ij[c, l1 m1] G_i[c, l2 m2]
    if k < L: V^k[c', l3 m] = sum_{c, q} Wmix_l3[c', c P_l3 + q] T[c, q, m] / sqrt(C P_l3)
              (q runs over the paths ending in l3, in path order)
    s     = scalar (l3 = 0) outputs T[c, q, 0], index c P_0 + q
    x^k   = (x^{k-1} + fc * MLP_k([x^{k-1}, s])) / sqrt(2)
  E_ij = MLP_E(x^L) (SiLU hidden layers, linear 1-wide output)
  E_i  = sigma_{Z_i} sum_j E_ij + mu_{Z_i},   E = sum_i E_i
Linear layers are bias-free, y = W x / sqrt(fan_in); latent MLPs apply
SiLU(z) = z / (1 + exp(-z)) after every layer.  Only l3 = 0 outputs of the last
layer are formed.  Forces come from torch.autograd in float64.
"""
import math

import numpy as np
import torch

from .blob import read_blob
from .neighbors import pairs_auto, pairs_cells, wrap_positions
from .sph import coupling_paths, real_cg, sh_real

F64 = torch.float64


def silu(z):
    return z * torch.sigmoid(z)


def bessel(d, r_cut, n_bessel):
    k = torch.arange(1, n_bessel + 1, dtype=F64)
    return math.sqrt(2.0 / r_cut) * torch.sin(k[None, :] * math.pi * d[:, None] / r_cut) / d[:, None]


def envelope(d, r_cut, p=6):
    """Polynomial cutoff u(x) = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1) - p(p+1)/2 x^(p+2)."""
    x = d / r_cut
    a = (p + 1) * (p + 2) / 2.0
    b = p * (p + 2.0)
    c = p * (p + 1) / 2.0
    return 1.0 - a * x ** p + b * x ** (p + 1) - c * x ** (p + 2)


class OracleModel:
    """emulate: None (exact FP64), "bf16", "fp16" or "fp16split".  With
    emulation, every per-pair GEMM (two-body, embedding, env, mixing, latent
    and energy hidden layers) rounds its input and its pre-scaled weight
    matrix (1/sqrt(fan_in), and 1/sqrt(nu) for env, folded in first) to that
    type and accumulates in FP64: the operand precision of the tensor-core
    path, used to check that path separately from the sensitivity of the
    model to rounding.  "fp16split" is "fp16" with the two-body MLP and the
    energy hidden layer left unrounded (the tensor-core path splits their
    operands into two FP16 parts, which carry about 22 bits).  In every
    emulation mode the per-pair values that the tensor-core path keeps in
    FP16 between its passes (x^k and the tensor-product scalars of layers
    k < L, V^k) are rounded to FP16 in the forward direction only (their
    gradients stay FP32 there).  The energy output layer, tensor products and
    all elementwise steps stay FP64."""

    def __init__(self, blob, emulate=None):
        cfg, w, names = read_blob(blob)
        self.cfg = cfg
        self.names = names
        self.w = {k: torch.tensor(v, dtype=F64) for k, v in w.items()}
        self.lmax = cfg["l_max"]
        self.L = cfg["n_layers"]
        self.C = cfg["n_channels"]
        self.S = cfg["n_species"]
        self.rc = cfg["r_cut"]
        self.nu = cfg["avg_num_neighbors"]
        self.paths = coupling_paths(self.lmax)
        self.cg = {p: torch.tensor(real_cg(*p), dtype=F64) for p in self.paths}
        if cfg["poly_p"] != 6:
            raise ValueError("poly_p = 6 only")
        if emulate not in (None, "bf16", "fp16", "fp16split"):
            raise ValueError("emulate must be None, 'bf16', 'fp16' or 'fp16split'")
        self.emulate = emulate
        self._qdt = {"bf16": torch.bfloat16, "fp16": torch.float16, "fp16split": torch.float16}.get(emulate)
        self._split = emulate == "fp16split"

    def _q(self, x):
        return x if self._qdt is None else x.to(self._qdt).to(F64)

    def _qs(self, x):
        """Emulation: FP16 storage of a forward value (gradient unchanged)."""
        if self._qdt is None:
            return x
        return x + (x.to(torch.float16).to(F64) - x).detach()

    def _qlin(self, x, W, extra=1.0):
        """Linear layer; in emulation mode the GEMM operands are rounded."""
        if self._qdt is None:
            return self._lin(x, W)
        s = extra / math.sqrt(W.shape[1])
        return self._q(x) @ self._q(W * s).T

    # ------------------------------------------------------------------ helpers
    def params(self):
        """Trainable tensors in blob order (a fresh leaf copy each call)."""
        return {k: self.w[k].clone() for k in self.names}

    @staticmethod
    def _lin(x, W):
        return x @ W.T / math.sqrt(W.shape[1])

    def _mlp(self, x, Ws, last_act=True, exact=False):
        for k, W in enumerate(Ws):
            x = self._lin(x, W) if exact else self._qlin(x, W)
            if last_act or k + 1 < len(Ws):
                x = silu(x)
        return x

    # ------------------------------------------------------------------ model
    def atom_energies(self, pos, species, lengths, pairs, w=None):
        """Per-atom energies E_i (torch float64, differentiable w.r.t. pos and w).

        pos: (N,3) float64 tensor; species: (N,) int; lengths: (3,) box edges;
        pairs: (i, j, n) integer arrays from the neighbour list of the same
        positions.
        """
        w = self.w if w is None else w
        cfg = self.cfg
        N = pos.shape[0]
        L = torch.tensor(np.array(lengths, dtype=np.float64))
        i = torch.as_tensor(np.asarray(pairs[0]), dtype=torch.int64)
        j = torch.as_tensor(np.asarray(pairs[1]), dtype=torch.int64)
        n = torch.as_tensor(np.asarray(pairs[2]), dtype=F64)
        Z = torch.as_tensor(np.asarray(species), dtype=torch.int64)
        sig = torch.tensor(cfg["sigma"], dtype=F64)[Z]
        mu = torch.tensor(cfg["mu"], dtype=F64)[Z]
        if i.shape[0] == 0:                     # no pairs: E_i = mu_Z (+ 0 * r for autograd)
            return mu + 0.0 * pos.sum(1)
        # wrapping is a constant shift per atom: gradients flow to pos unchanged
        with torch.no_grad():
            shift = torch.as_tensor(wrap_positions(pos.detach().numpy(), lengths)) - pos.detach()
        wpos = pos + shift
        delta = (wpos[j] - wpos[i]) + n * L[None, :]
        d = torch.sqrt((delta * delta).sum(-1))
        u = delta / d[:, None]
        B = bessel(d, self.rc, cfg["n_bessel"])
        fc = envelope(d, self.rc, cfg["poly_p"])
        Y = sh_real(u, self.lmax)
        S, C, lmax = self.S, self.C, self.lmax
        P = i.shape[0]
        onehot = torch.eye(S, dtype=F64)
        h = torch.cat([onehot[Z[i]], onehot[Z[j]], B], dim=1)
        nlat = len(cfg["latent"])
        x = self._qs(fc[:, None] * self._mlp(h, [w[f"twobody.{k}"] for k in range(nlat)], exact=self._split))
        w0 = self._qlin(x, w["embed"]).view(P, C, lmax + 1)
        V = [w0[:, :, l, None] * Y[l][:, None, :] for l in range(lmax + 1)]
        for layer in range(1, self.L + 1):
            last = layer == self.L
            if self._qdt is None:
                e = self._lin(x, w[f"layer{layer}.env"]) / math.sqrt(self.nu)   # (P, C)
            else:
                e = self._qlin(x, w[f"layer{layer}.env"], 1.0 / math.sqrt(self.nu))
            G = []
            for l in range(lmax + 1):
                contrib = e[:, :, None] * Y[l][:, None, :]
                Gl = torch.zeros((N, C, 2 * l + 1), dtype=F64).index_add(0, i, contrib)
                G.append(Gl[i])
            T = {}
            for p in self.paths:
                l1, l2, l3 = p
                if last and l3 != 0:
                    continue
                T[p] = torch.einsum("abc,pna,pnb->pnc", self.cg[p], V[l1], G[l2])
            scal = [p for p in self.paths if p[2] == 0]
            s = torch.stack([T[p][:, :, 0] for p in scal], dim=2).reshape(P, C * len(scal))
            if not last:
                newV = []
                for l3 in range(lmax + 1):
                    ps = [p for p in self.paths if p[2] == l3]
                    Tl = torch.stack([T[p] for p in ps], dim=2)        # (P, C, Pl, 2l3+1)
                    Tl = Tl.reshape(P, C * len(ps), 2 * l3 + 1)
                    Wm = w[f"layer{layer}.mix{l3}"]
                    if self._qdt is None:
                        newV.append(torch.einsum("oi,pim->pom", Wm, Tl) / math.sqrt(C * len(ps)))
                    else:
                        Wq = self._q(Wm / math.sqrt(C * len(ps)))
                        newV.append(torch.einsum("oi,pim->pom", Wq, self._q(Tl)))
                V = [self._qs(v) for v in newV]
            if not last:
                s = self._qs(s)
            m = self._mlp(torch.cat([x, s], dim=1),
                          [w[f"layer{layer}.latent.{k}"] for k in range(nlat)])
            x = (x + fc[:, None] * m) / math.sqrt(2.0)
            if not last:
                x = self._qs(x)
        ne = len(cfg["energy"])
        hdn = self._mlp(x, [w[f"energy.{k}"] for k in range(ne)], exact=self._split)
        Eij = self._lin(hdn, w["energy.out"])[:, 0]
        Esum = torch.zeros(N, dtype=F64).index_add(0, i, Eij)
        return sig * Esum + mu

    def energy_forces(self, pos, species, lengths, pairs=None, w=None):
        """Return (E float, F (N,3) ndarray, E_i (N,) ndarray, pairs)."""
        pos = np.asarray(pos, dtype=np.float64)
        if pairs is None:
            pairs = pairs_auto(pos, lengths, self.rc)
        r = torch.tensor(pos, dtype=F64, requires_grad=True)
        Ei = self.atom_energies(r, species, lengths, pairs, w=w)
        E = Ei.sum()
        (g,) = torch.autograd.grad(E, r)
        return float(E.detach()), (-g).numpy(), Ei.detach().numpy(), pairs

    # ------------------------------------------------- local (sampled) evaluation
    def local_energy_force(self, pos, species, lengths, k):
        """E_k and F_k of one atom in a large periodic system, from its 2 r_cut
        neighbourhood only (exact because E_i depends only on atoms within
        r_cut of i).  Needs L > 4 r_cut + 1 on every axis."""
        L = np.asarray(lengths, dtype=np.float64)
        rc = self.rc
        assert np.all(L > 4 * rc + 1.0)
        w = wrap_positions(np.asarray(pos, np.float64), L)
        dvec = w - w[k][None, :]
        dvec -= np.round(dvec / L[None, :]) * L[None, :]
        dist = np.sqrt((dvec * dvec).sum(1))
        sel = np.nonzero(dist < 2 * rc + 0.5)[0]
        kk = int(np.nonzero(sel == k)[0][0])
        big = np.array([1000.0, 1000.0, 1000.0])
        cpos = dvec[sel] + 500.0
        csp = np.asarray(species)[sel]
        pairs = pairs_auto(cpos, big, rc)
        r = torch.tensor(cpos, dtype=F64, requires_grad=True)
        Ei = self.atom_energies(r, csp, big, pairs)
        inner = torch.as_tensor(dist[sel] < rc)
        inner[kk] = True
        Esub = Ei[inner].sum()
        (g,) = torch.autograd.grad(Esub, r)
        return float(Ei[kk].detach()), -g[kk].numpy()
