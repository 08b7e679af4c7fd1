"""Tolerances of the tensor-core path against the emulating oracle, derived
from a stated model of the GPU's own arithmetic (test infrastructure).

The emulating oracle (oracle/model.py, emulate=...) rounds the same operands
and stored values as the tensor-core kernels, but it rounds FP64 values while
the kernels round their FP32 values.  Where the two lie on different sides of
a rounding boundary, the rounded values differ by one unit in the last place;
those flips, and the FP32 arithmetic of what is not rounded, are the whole
difference between the two.  Their effect is estimated here with the oracle
alone, by a perturbation analysis: the oracle is evaluated again with every
value it rounds perturbed by the error the GPU carries into that rounding, and
the spread of the results is the scale of the GPU-vs-emulation difference.
The error model, per value:
  * SiLU(z) = z sigmoid(z), sigmoid through tanh.approx.f32: absolute error
    within |z| 2^-17.5 (the bound tests/test_gpu_umma.py checks on the
    passes' own SiLU), modelled as uniform in +-|z| 2^-17.5;
  * adjoint-GEMM gradient operands carry the SiLU derivative's error,
    (1 + |z|) 2^-17.5 against a derivative of order 1, and FP32 accumulation:
    relative, uniform in +-2^-15;
  * every other value about to be rounded (GEMM inputs, stored x^k, V^k and
    layer scalars) carries FP32 accumulation and FP32 geometry: relative,
    uniform in +-2^-22;
  * split-mode operands (two-body MLP and energy hidden layer: x = hi + lo
    with two FP16 parts, the lo x lo product dropped) carry a relative
    2^-22 and, where lo is FP16-subnormal (|lo| < 2^-14, spacing 2^-24), an
    absolute 2^-25: uniform in +-(2^-22 |a| + 2^-25), inputs and weights.
A bound is 8 times the root-mean-square deviation over the draws (a Gaussian
tail of 8 sigma, which leaves room for the few draws the estimate rests on),
plus a floor for the FP32 arithmetic of the steps that are not rounded at
all (tensor products, energy output layer, FP32 sums): 2^-22 of the sum of
|E_i| for the total energy, 2^-20 of max |E_i| per atom and 2^-20 of max
|F| for forces."""
import numpy as np
import torch

from oracle.model import OracleModel

F64 = torch.float64
SIGMOID_ABS = 2.0 ** -17.5


def perturbation_bounds(blob, mode, pos, species, lengths, pairs, draws=4, seed=0):
    """(E, F, E_i) of the emulating oracle and the bounds (dE, dF, dE_i) on
    the tensor-core path's deviation from them."""
    base = OracleModel(blob, emulate=mode)
    E0, F0, Ei0, _ = base.energy_forces(pos, species, lengths, pairs=pairs)
    sE, sF, sEi = [], [], []
    for k in range(draws):
        g = torch.Generator().manual_seed(seed + k)

        def u(shape):
            return torch.rand(shape, generator=g, dtype=F64) * 2.0 - 1.0

        m = OracleModel(blob, emulate=mode)
        m.perturb_silu = lambda z: u(z.shape) * z.abs() * SIGMOID_ABS
        m.perturb_grad = lambda v: v * (1.0 + u(v.shape) * 2.0 ** -15)
        m.perturb_value = lambda v: v * (1.0 + u(v.shape) * 2.0 ** -22)
        m.perturb_split = lambda a: a + u(a.shape) * (a.abs() * 2.0 ** -22 + 2.0 ** -25)
        E, F, Ei, _ = m.energy_forces(pos, species, lengths, pairs=pairs)
        sE.append(E - E0)
        sF.append(F - F0)
        sEi.append(Ei - Ei0)
    rms = lambda a: np.sqrt(np.mean(np.square(np.asarray(a)), axis=0))
    dE = 8.0 * float(rms(sE)) + 2.0 ** -22 * float(np.abs(Ei0).sum())
    dEi = 8.0 * float(rms(sEi).max()) + 2.0 ** -20 * float(np.abs(Ei0).max())
    dF = 8.0 * float(rms(sF).max()) + 2.0 ** -20 * float(np.abs(F0).max())
    return (E0, F0, Ei0), (dE, dF, dEi)
