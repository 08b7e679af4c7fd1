"""Loss, weight gradient, Adam and the SAM step (oracle).

Eq. 3 (SAM): w <- w - eta grad L(w') at w' = w + rho grad L(w) / ||grad L(w)||.
Base optimizer Adam with (beta1, beta2) = (0.9, 0.999) (Table 5), eps = 1e-8.
Loss (Table 5 "per atom MSE", with the energy:force weights as arguments):
    L = (w_E / B) sum_b ((E_b - E*_b) / N_b)^2
        + (w_F / (3 sum_b N_b)) sum_b sum_i |F_bi - F*_bi|^2
Sharpness (Eq. 2) and the loss landscape of Sec. 5.4 (Table 4, Fig. 5): the
loss at w + eps for sampled eps of norm rho, and along one direction.
Readings: the trainable vector is every weight matrix of the blob flattened
row-major in blob order (sigma_Z, mu_Z fixed); ||.|| is the global L2 norm; if
||grad L|| = 0 the ascent step is zero.  The force term's weight gradient is a
double backward through torch.autograd in float64.
"""
import math

import numpy as np
import torch

from .neighbors import pairs_auto

F64 = torch.float64


def flat_params(model):
    return torch.cat([model.w[k].reshape(-1) for k in model.names]).clone()


def _unflat(model, vec):
    out, off = {}, 0
    for k in model.names:
        shp = model.w[k].shape
        n = shp[0] * shp[1]
        out[k] = vec[off:off + n].view(shp)
        off += n
    return out


def loss_and_grad(model, wvec, batch, w_energy=1.0, w_force=100.0, need_grad=True):
    """batch: list of dicts {pos, species, lengths, e_target, f_target[, pairs]}.

    Returns (loss float, grad ndarray or None)."""
    vec = torch.as_tensor(np.asarray(wvec), dtype=F64).clone().requires_grad_(need_grad)
    w = _unflat(model, vec)
    B = len(batch)
    n_tot = sum(len(s["species"]) for s in batch)
    le = torch.zeros((), dtype=F64)
    lf = torch.zeros((), dtype=F64)
    for s in batch:
        pairs = s.get("pairs")
        if pairs is None:
            pairs = pairs_auto(s["pos"], s["lengths"], model.rc)
        r = torch.tensor(np.asarray(s["pos"]), dtype=F64, requires_grad=True)
        Ei = model.atom_energies(r, s["species"], s["lengths"], pairs, w=w)
        E = Ei.sum()
        (g,) = torch.autograd.grad(E, r, create_graph=need_grad)
        F = -g
        nb = r.shape[0]
        le = le + ((E - float(s["e_target"])) / nb) ** 2
        ft = torch.as_tensor(np.asarray(s["f_target"], dtype=np.float64))
        lf = lf + ((F - ft) ** 2).sum()
    loss = w_energy * le / B + w_force * lf / (3.0 * n_tot)
    if not need_grad:
        return float(loss.detach()), None
    (gw,) = torch.autograd.grad(loss, vec)
    return float(loss.detach()), gw.numpy()


def loss_scan(model, w, dirs, scales, batch, w_energy=1.0, w_force=100.0):
    """L(w + scales[k] d_k) for every point k: the loss landscape around w that
    the sharpness of Eq. 2 is defined on.  dirs: one row per point, or one row
    shared by every point.  Returns an ndarray of losses."""
    w = np.asarray(w, dtype=np.float64)
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    scales = np.asarray(scales, dtype=np.float64).reshape(-1)
    if dirs.shape[0] not in (1, scales.shape[0]):
        raise ValueError("one direction per scale, or one direction for all")
    out = []
    for k, sk in enumerate(scales):
        d = dirs[k] if dirs.shape[0] > 1 else dirs[0]
        out.append(loss_and_grad(model, w + sk * d, batch, w_energy, w_force, need_grad=False)[0])
    return np.array(out)


def sharpness(model, w, eps, batch, w_energy=1.0, w_force=100.0):
    """Eq. 2, max over ||eps|| <= rho of L(w + eps) - L(w), estimated as in
    Sec. 5.4 (Table 4) by the largest value over the given samples eps_k
    (rows of eps)."""
    eps = np.atleast_2d(np.asarray(eps, dtype=np.float64))
    base = loss_and_grad(model, w, batch, w_energy, w_force, need_grad=False)[0]
    return float(np.max(loss_scan(model, w, eps, np.ones(eps.shape[0]), batch, w_energy, w_force)) - base)


def adam_update(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step; returns (w, m, v, t) as new arrays."""
    t = t + 1
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    w = w - lr * mhat / (np.sqrt(vhat) + eps)
    return w, m, v, t


def sam_step(model, w, batch, rho, lr, state, w_energy=1.0, w_force=100.0):
    """One SAM step (Eq. 3) with Adam as the base optimizer.

    state = (m, v, t).  Returns (w_new, state_new, loss_at_w, loss_at_w_prime,
    eps_vector)."""
    w = np.asarray(w, dtype=np.float64)
    l0, g = loss_and_grad(model, w, batch, w_energy, w_force)
    gn = math.sqrt(float(np.dot(g, g)))
    eps = (rho / gn) * g if gn > 0 else np.zeros_like(g)
    l1, g2 = loss_and_grad(model, w + eps, batch, w_energy, w_force)
    m, v, t = state
    w_new, m, v, t = adam_update(w, g2, m, v, t, lr)
    return w_new, (m, v, t), l0, l1, eps
