"""Seeded initial parameters of a three-layer perceptron (nin -> nh -> nh ->
nout): weights uniform in +-1/sqrt(fan_in), biases zero, packed as
W1[nh][nin], b1, W2[nh][nh], b2, W3[nout][nh], b3.  A random draw only."""
from __future__ import annotations

import math

import numpy as np


def mlp_init(nin, nh, nout, seed=0):
    rng = np.random.Generator(np.random.PCG64([seed, nin, nh, nout]))
    parts = []
    for rows, cols in ((nh, nin), (nh, nh), (nout, nh)):
        lim = 1.0 / math.sqrt(cols)
        parts.append(rng.uniform(-lim, lim, size=rows * cols))
        parts.append(np.zeros(rows))
    return np.concatenate(parts)
