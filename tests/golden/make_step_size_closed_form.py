"""Writes step_size_closed_form.txt: the step-size constant of the 64x64
binary denoising model from its closed form (Sec. 3.2 and Sec. 4.3).

The potential matrix of a 4-connected H x W grid with unit weights and Potts
coupling c [l != m] (L = 2) is A (x) mu.  On the tangent space of the simplex
product mu acts as -c, and the spectrum of the grid adjacency A is
{2cos(a pi/(H+1)) + 2cos(b pi/(W+1))}, symmetric about zero (the grid is
bipartite), so Lambda = c (2cos(pi/(H+1)) + 2cos(pi/(W+1))) and
eta = 1/(1 + Lambda).  The library takes float32 inputs, so c is float32(0.8).

Run: python tests/golden/make_step_size_closed_form.py
"""
import math
import os

import numpy as np

H = W = 64
c = float(np.float32(0.8))
lam = c * (2 * math.cos(math.pi / (H + 1)) + 2 * math.cos(math.pi / (W + 1)))
eta = 1.0 / (1.0 + lam)

HEADER = """# Step-size constant of the 64x64 binary denoising model (Sec. 3.2: the highest
# eigenvalue of the constant Hessian -- the "potential matrix" -- is a valid
# Lipschitz constant; Sec. 4.3 sets d to it), read on the tangent space of the
# simplex product.
#
# Model: 4-connected 64x64 grid, unit edge weights, Potts mu = 0.8 [l != m], L = 2.
# The potential matrix is A (x) mu with A the grid adjacency.  On the tangent
# space mu acts as -0.8, and the grid adjacency spectrum is
# {2cos(a pi/65) + 2cos(b pi/65) : a, b = 1..64}, symmetric about 0 (the grid
# is bipartite), so
#   Lambda = 0.8 * (2cos(pi/65) + 2cos(pi/65)),   eta = 1 / (1 + Lambda).
# The library takes float32 inputs, so the coupling is float32(0.8) =
# 0.800000011920928955078125; the constant below uses that value.
# Written by make_step_size_closed_form.py (IEEE double, math.cos).
"""

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "step_size_closed_form.txt")
    with open(out, "w") as f:
        f.write(HEADER)
        f.write(f"H {H}\nW {W}\ncoupling {c:.15g}\nLambda {lam!r}\neta {eta!r}\n")
