"""Test helpers: the synthetic projectors rebuilt from their analytic form,
independently of the generator's tables."""
import math

import numpy as np

from paper_2302_09708_gb300 import synth


def analytic_projectors(s, k=(0.0, 0.0, 0.0)):
    """Each atom's projectors from their analytic form, g_0 Y_00 and g_1 Y_1m
    (m-order y, z, x) with g = exp(-r^2 / 2 sigma^2), cut off at RC, summed
    over the 27 nearest lattice images with Bloch weights exp(i k.T) and
    normalised to h^3 sum |chi|^2 = 1 (the phases have modulus one).  Returns a
    list of (Nd x 4 complex matrix, gammas) per atom."""
    k = np.asarray(k, dtype=np.float64)
    nx, ny, nz = s.shape
    L = np.array(s.shape, dtype=np.float64) * s.h
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.stack([ix.ravel() * s.h, iy.ravel() * s.h, iz.ravel() * s.h], axis=1)
    out = []
    y00, y1 = 0.5 / math.sqrt(math.pi), math.sqrt(3.0 / (4.0 * math.pi))
    for J in range(s.natoms):
        real = np.zeros((s.nd, 4))
        bloch = np.zeros((s.nd, 4), dtype=np.complex128)
        for tx in (-1, 0, 1):
            for ty in (-1, 0, 1):
                for tz in (-1, 0, 1):
                    t = np.array([tx, ty, tz], dtype=np.float64)
                    if any(t[d] != 0 and s.bc[d] != synth.PERIODIC for d in range(3)):
                        continue
                    T = t * L
                    dvec = r - s.positions[J] - T
                    r2 = np.sum(dvec * dvec, axis=1)
                    g = np.where(r2 <= synth.RC ** 2, np.exp(-r2 / (2 * synth.SIGMA ** 2)), 0.0)
                    cols = np.stack([g * y00, g * y1 * dvec[:, 1], g * y1 * dvec[:, 2],
                                     g * y1 * dvec[:, 0]], axis=1)
                    real += cols
                    bloch += cols * np.exp(1j * float(k @ T))
        norm = np.sqrt(s.h ** 3 * np.sum(real * real, axis=0))
        out.append((bloch / norm[None, :], s.gamma[int(s.proj_ptr[J]):int(s.proj_ptr[J + 1])]))
    return out
