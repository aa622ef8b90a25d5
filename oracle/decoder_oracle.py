"""FP64 reference of the learned initialiser's layers (transposed 1-D convolution, GELU).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Layer definition (stride 2, kernel 9, padding 4, output padding 1; output
length twice the input length):

    y[b][co][t] = bias[co] + sum_{ci, u, k : t = 2u - 4 + k} x[b][ci][u] W[ci][co][k]

GELU(z) = z/2 (1 + erf(z / sqrt 2)).  ``conv_transpose`` evaluates the
definition with torch's float64 transposed convolution (a library primitive);
``conv_transpose_direct`` is the same sum written out term by term, for tiny
sizes, and pins the first.
"""

from __future__ import annotations

import math

import numpy as np
import torch

KERNEL = 9
STRIDE = 2
PAD = 4


def conv_transpose(x: torch.Tensor, w: torch.Tensor, bias: torch.Tensor) -> torch.Tensor:
    """x [B][Ci][T], w [Ci][Co][9], bias [Co] (any float dtype) -> float64 [B][Co][2T]."""
    return torch.nn.functional.conv_transpose1d(x.double(), w.double(), bias.double(), stride=STRIDE,
                                                padding=PAD, output_padding=1)


def conv_transpose_direct(x: np.ndarray, w: np.ndarray, bias: np.ndarray) -> np.ndarray:
    """The defining sum, term by term (tiny sizes only)."""
    B, Ci, T = x.shape
    Co = w.shape[1]
    y = np.zeros((B, Co, 2 * T)) + bias[None, :, None]
    for b in range(B):
        for ci in range(Ci):
            for u in range(T):
                for k in range(KERNEL):
                    t = STRIDE * u - PAD + k
                    if 0 <= t < 2 * T:
                        y[b, :, t] += x[b, ci, u] * w[ci, :, k]
    return y


def gelu(z: torch.Tensor) -> torch.Tensor:
    z = z.double()
    return 0.5 * z * (1.0 + torch.erf(z / math.sqrt(2.0)))
