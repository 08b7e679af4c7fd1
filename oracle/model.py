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
  With the blob's parity flag set (full O(3)), features are irreps (l, s),
  s = 1 for the parity opposite to Y_l's (pseudotensors); V^0 is all s = 0, the
  paths of a layer run from every input irrep (l1, s1) present through Y_l2 to
  l3 with l1 + l2 + l3 of either parity, landing in s3 = (l1 + s1 + l2 + l3)
  mod 2; each output irrep (l3, s3) is mixed by its own matrix (mix{l3} for
  s3 = 0, mix{l3}p for s3 = 1) over its paths, ordered by s1, then l1, then
  l2; the latent MLP takes the true scalars (0, 0) only.  Without the flag
  only paths with s1 = s3 = 0 exist (l1 + l2 + l3 even), which is the model
  above.
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


def round_to(x, dtype):
    """x rounded to the floating-point type dtype (round to nearest, ties to
    even, as every conversion here does), returned in float64."""
    return x.to(dtype).to(F64)


class RoundedLinear(torch.autograd.Function):
    """Emulated tensor-core GEMM y = q(x) q(Ws)^T, accumulated in float64, with
    q(.) the operand rounding and Ws the weight matrix with its scale folded
    in.  Its adjoint (the input-gradient GEMM) rounds its operands the same
    way: dx = q(dy) q(Ws).  The weight gradient is left exact."""

    @staticmethod
    def forward(ctx, x, Ws, q_x, q_w, q_adj):
        xq, Wq = q_x(x), q_w(Ws)
        ctx.save_for_backward(xq, Wq)
        ctx.q_adj = q_adj
        return xq @ Wq.T

    @staticmethod
    def backward(ctx, g):
        xq, Wq = ctx.saved_tensors
        return ctx.q_adj(g) @ Wq, g.T @ xq, None, None, None


class OracleModel:
    """emulate: None (exact FP64), "bf16", "fp16" or "fp16split".

    Emulation models the operand precision of the tensor-core path, so that
    the kernels can be checked separately from the sensitivity of the model to
    rounding:
      * every per-pair GEMM (two-body, embedding, env, mixing, latent and
        energy hidden layers) is a RoundedLinear: its input and its pre-scaled
        weight matrix (1/sqrt(fan_in), and 1/sqrt(nu) for env, folded in
        first) are rounded to op_dtype and accumulated in FP64, and its
        adjoint GEMM rounds the incoming gradient to op_dtype as well;
      * "fp16split" is "fp16" with the GEMMs of the groups in exact_groups
        (the two-body MLP and the energy hidden layer) left unrounded: the
        tensor-core path splits their operands into two FP16 parts, which
        carry about 22 bits;
      * the per-pair values that the tensor-core path keeps between its passes
        (x^k and the tensor-product scalars of layers k < L, and V^k) are
        rounded to store_dtype (FP16) in the forward direction only: the
        gradient passes through unchanged (straight-through), as the path keeps
        gradients in FP32;
      * the energy output layer, the tensor products and every elementwise
        step stay FP64.
    op_dtype, adj_dtype, store_dtype and exact_groups are plain attributes, so
    that tests can substitute them (float64 makes every rounding an identity).
    perturb_silu(z), perturb_value(x), perturb_grad(g) and perturb_split(a),
    None by default, are hooks for a perturbation analysis: the first returns
    an additive perturbation of SiLU(z), the second a perturbed copy of a
    forward value about to be rounded (a GEMM input or a stored value), the
    third a perturbed copy of an adjoint-GEMM gradient operand about to be
    rounded, the fourth a perturbed copy of an operand (input or pre-scaled
    weight) of a GEMM of the exact groups.  Rounded weights are never
    perturbed; the hooks change forward values only (gradients pass
    through)."""

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
        self.o3 = cfg.get("parity", 0) == 1
        self.paths = coupling_paths(self.lmax)
        self.cg = {p: torch.tensor(real_cg(*p), dtype=F64)
                   for p in coupling_paths(self.lmax, parity="all" if self.o3 else "even")}
        if cfg["poly_p"] != 6:
            raise ValueError("poly_p = 6 only")
        if emulate not in (None, "bf16", "fp16", "fp16split"):
            raise ValueError("emulate must be None, 'bf16', 'fp16' or 'fp16split'")
        self.emulate = emulate
        self.op_dtype = {"bf16": torch.bfloat16, "fp16": torch.float16, "fp16split": torch.float16}.get(emulate)
        self.adj_dtype = self.op_dtype
        self.store_dtype = torch.float16 if emulate else None
        self.exact_groups = {"twobody", "energy"} if emulate == "fp16split" else set()
        self.perturb_silu = None
        self.perturb_value = None
        self.perturb_grad = None
        self.perturb_split = None

    def _pre(self, x, hook=None):
        """A value about to be rounded, with a perturbation hook applied."""
        hook = self.perturb_value if hook is None else hook
        if hook is None:
            return x
        with torch.no_grad():
            return hook(x.detach())

    def _q_op(self, x):
        return round_to(self._pre(x), self.op_dtype)

    def _q_w(self, W):
        return round_to(W, self.op_dtype)

    def _q_adj(self, g):
        if self.perturb_grad is not None:
            g = self._pre(g, self.perturb_grad)
        return round_to(g, self.adj_dtype)

    def _qs(self, x):
        """Emulation: storage of a forward value in store_dtype (gradient
        passes through unchanged)."""
        if self.store_dtype is None:
            return x
        return x + (round_to(self._pre(x), self.store_dtype) - x).detach()

    def _act(self, z):
        a = silu(z)
        if self.perturb_silu is not None:
            with torch.no_grad():
                d = self.perturb_silu(z.detach())
            a = a + d
        return a

    def _qlin(self, x, W, extra=1.0, group=None):
        """Linear layer; emulated as a RoundedLinear unless exact."""
        if self.op_dtype is None or group in self.exact_groups:
            if self.perturb_split is not None and group in self.exact_groups:
                s = extra / math.sqrt(W.shape[1])
                with torch.no_grad():
                    dx = self.perturb_split(x.detach()) - x.detach()
                    Ws = W.detach() * s
                    dW = self.perturb_split(Ws) - Ws
                return (x + dx) @ (W * s + dW).T
            return self._lin(x, W) if extra == 1.0 else self._lin(x, W) * extra
        s = extra / math.sqrt(W.shape[1])
        return RoundedLinear.apply(x, W * s, self._q_op, self._q_w, self._q_adj)

    # ------------------------------------------------------------------ helpers
    def params(self):
        """Trainable tensors in blob order (a fresh leaf copy each call)."""
        return {k: self.w[k].clone() for k in self.names}

    @staticmethod
    def _lin(x, W):
        return x @ W.T / math.sqrt(W.shape[1])

    def _mlp(self, x, Ws, last_act=True, group=None):
        for k, W in enumerate(Ws):
            x = self._qlin(x, W, group=group)
            if last_act or k + 1 < len(Ws):
                x = self._act(x)
        return x

    def layer_paths(self, irreps):
        """{(l3, s3): [(l1, s1, l2), ...]} for a layer whose input features
        carry the irreps in `irreps`; paths in (s1, l1, l2) order."""
        out = {}
        for s1 in (0, 1):
            for l1 in range(self.lmax + 1):
                if (l1, s1) not in irreps:
                    continue
                for l2 in range(self.lmax + 1):
                    for l3 in range(abs(l1 - l2), min(l1 + l2, self.lmax) + 1):
                        s3 = (l1 + s1 + l2 + l3) % 2
                        if not self.o3 and (s1 or s3):
                            continue
                        out.setdefault((l3, s3), []).append((l1, s1, l2))
        return out

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
        x = self._qs(fc[:, None] * self._mlp(h, [w[f"twobody.{k}"] for k in range(nlat)], group="twobody"))
        w0 = self._qlin(x, w["embed"], group="embed").view(P, C, lmax + 1)
        # features: irrep (l, s) -> (P, C, 2l + 1)
        V = {(l, 0): w0[:, :, l, None] * Y[l][:, None, :] for l in range(lmax + 1)}
        for layer in range(1, self.L + 1):
            last = layer == self.L
            if self.op_dtype is None:
                e = self._lin(x, w[f"layer{layer}.env"]) / math.sqrt(self.nu)   # (P, C)
            else:
                e = self._qlin(x, w[f"layer{layer}.env"], 1.0 / math.sqrt(self.nu), group="env")
            G = []
            for l in range(lmax + 1):
                contrib = e[:, :, None] * Y[l][:, None, :]
                Gl = torch.zeros((N, C, 2 * l + 1), dtype=F64).index_add(0, i, contrib)
                G.append(Gl[i])
            T = {}                                    # output irrep -> [per-path (P, C, 2 l3 + 1)]
            for (l3, s3), plist in self.layer_paths(set(V)).items():
                if last and (l3, s3) != (0, 0):
                    continue
                T[(l3, s3)] = [torch.einsum("abc,pna,pnb->pnc", self.cg[(l1, l2, l3)], V[(l1, s1)], G[l2])
                               for (l1, s1, l2) in plist]
            s = torch.stack([t[:, :, 0] for t in T[(0, 0)]], dim=2).reshape(P, C * len(T[(0, 0)]))
            if not last:
                newV = {}
                for (l3, s3), tl in T.items():
                    Tl = torch.stack(tl, dim=2)                       # (P, C, Pl, 2l3+1)
                    Tl = Tl.reshape(P, C * len(tl), 2 * l3 + 1)
                    Wm = w[f"layer{layer}.mix{l3}" + ("p" if s3 else "")]
                    if self.op_dtype is None:
                        newV[(l3, s3)] = torch.einsum("oi,pim->pom", Wm, Tl) / math.sqrt(C * len(tl))
                    else:
                        # one GEMM over the (pair, m) rows of the K = C P_l3 inputs
                        nm = 2 * l3 + 1
                        rows = Tl.permute(0, 2, 1).reshape(P * nm, C * len(tl))
                        out = self._qlin(rows, Wm, group="mix")
                        newV[(l3, s3)] = out.reshape(P, nm, C).permute(0, 2, 1)
                V = {key: self._qs(v) for key, v in newV.items()}
            if not last:
                s = self._qs(s)
            m = self._mlp(torch.cat([x, s], dim=1),
                          [w[f"layer{layer}.latent.{k}"] for k in range(nlat)], group="latent")
            x = (x + fc[:, None] * m) / math.sqrt(2.0)
            if not last:
                x = self._qs(x)
        ne = len(cfg["energy"])
        hdn = self._mlp(x, [w[f"energy.{k}"] for k in range(ne)], group="energy")
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
