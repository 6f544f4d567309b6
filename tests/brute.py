"""Independent O(N^2) brute force for tiny grids (test infrastructure).

A second, deliberately different implementation of the same discrete operator
the oracle evaluates, used only to pin the oracle: instead of interpolating the
field at every quadrature node, it tabulates the kernel value K(d) for every
grid displacement d (its own quadrature nodes from numpy's Gauss-Legendre
routine, its own hat-function weights) and sums every output point against
every input point.  Periodic axes sum all images of the displacement; other
axes are zero-extended (Sec 3.5).  Works on complex input (complex-step checks).
"""
from __future__ import annotations

import math

import numpy as np


def angular_rule(radius: float, nmu: int = 0, ntheta: int = 0):
    """Trapezoid in theta x Gauss-Legendre in cos(phi) (Sec 3.5 reading)."""
    if nmu <= 0:
        nmu = max(8, math.ceil(2 * math.pi * radius))
    if ntheta <= 0:
        ntheta = -(-2 * nmu // 4) * 4
    mu, wmu = np.polynomial.legendre.leggauss(nmu)
    th = (np.arange(ntheta) + 0.5) * 2 * np.pi / ntheta
    M, T = np.meshgrid(mu, th, indexing="ij")
    W = np.repeat(wmu[:, None], ntheta, 1) * (2 * np.pi / ntheta)
    s = np.sqrt(1 - M ** 2)
    u = np.stack([np.cos(T) * s, np.sin(T) * s, M], -1).reshape(-1, 3)
    return u, W.reshape(-1)


def radial_rule(a: float, b: float, nr: int = 0):
    if nr <= 0:
        nr = max(4, math.ceil(2 * (b - a)))
    x, w = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * (b - a) * x + 0.5 * (b + a)
    return r, 0.5 * (b - a) * w * r * r


def nodes(kind: str, R: float, r_in: float = 0.0, nmu=0, ntheta=0, nr=0):
    """('shell' | 'ball' | 'thick') -> positions p[n,3], weights w[n], units u[n,3]."""
    if kind == "shell":
        u, w = angular_rule(R, nmu, ntheta)
        return R * u, R * R * w, u
    u, wa = angular_rule(R, nmu, ntheta)
    r, wr = radial_rule(0.0 if kind == "ball" else r_in, R, nr)
    p = (r[:, None, None] * u[None, :, :]).reshape(-1, 3)
    w = (wr[:, None] * wa[None, :]).reshape(-1)
    uu = np.broadcast_to(u[None], (len(r),) + u.shape).reshape(-1, 3)
    return p, w, uu


def kernel_table(p, w, u, reach: int, vector: bool = False):
    """K(d) = sum_q w_q hat(d - p_q) [u_q] for integer d in [-reach, reach]^3,
    hat(v) = prod_axes max(0, 1 - |v|) (the trilinear weight)."""
    d = np.arange(-reach, reach + 1)
    out_shape = (2 * reach + 1,) * 3
    K = np.zeros(out_shape + ((3,) if vector else ()))
    for q in range(len(w)):
        hx = np.maximum(0.0, 1 - np.abs(d - p[q, 0]))
        hy = np.maximum(0.0, 1 - np.abs(d - p[q, 1]))
        hz = np.maximum(0.0, 1 - np.abs(d - p[q, 2]))
        h3 = hz[:, None, None] * hy[None, :, None] * hx[None, None, :]   # [dz, dy, dx]
        if vector:
            K += w[q] * h3[..., None] * u[q][None, None, None, :]
        else:
            K += w[q] * h3
    return K


def dense_operator(K, reach, shape, periodic):
    """M[out, in] = K(r_in - r_out) summed over periodic images; shape = (nz, ny, nx),
    periodic = (px, py, pz).  K indexed [dz, dy, dx, ...]."""
    nz, ny, nx = shape
    pts = np.stack(np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"), -1).reshape(-1, 3)
    npts = len(pts)
    extra = K.shape[3:]
    M = np.zeros((npts, npts) + extra)
    dims = (nz, ny, nx)
    per = (periodic[2], periodic[1], periodic[0])
    images = []
    for ax in range(3):
        if per[ax]:
            m = reach // dims[ax] + 1
            images.append(range(-m, m + 1))
        else:
            images.append([0])
    for a, r_out in enumerate(pts):
        diff = pts - r_out                     # displacement in -> relative to out
        for iz in images[0]:
            for iy in images[1]:
                for ix in images[2]:
                    dd = diff + np.array([iz * nz, iy * ny, ix * nx])
                    ok = np.all(np.abs(dd) <= reach, axis=1)
                    idx = dd[ok] + reach
                    M[a, ok] += K[idx[:, 0], idx[:, 1], idx[:, 2]]
    return M


class BruteFMT:
    """Dense weighted-density operators for a small grid."""

    def __init__(self, shape, periodic, R, nmu=0, ntheta=0, nr=0):
        self.shape = shape
        self.periodic = periodic
        self.R = list(R)
        self.ops = []
        for r in self.R:
            reach = int(math.ceil(r)) + 1
            ps, ws, us = nodes("shell", r, nmu=nmu, ntheta=ntheta)
            pb, wb, ub = nodes("ball", r, nmu=nmu, ntheta=ntheta, nr=nr)
            M2 = dense_operator(kernel_table(ps, ws, us, reach), reach, shape, periodic)
            M3 = dense_operator(kernel_table(pb, wb, ub, reach), reach, shape, periodic)
            Mv = dense_operator(kernel_table(ps, ws, us, reach, vector=True), reach, shape, periodic)
            self.ops.append((M2, M3, Mv))

    def weighted(self, rho):
        """rho [s, nz, ny, nx] (real or complex) -> n [10, nz, ny, nx]."""
        N = int(np.prod(self.shape))
        out = np.zeros((10, N), dtype=np.result_type(rho.dtype, np.float64))
        for i, (M2, M3, Mv) in enumerate(self.ops):
            r = rho[i].reshape(N)
            R = self.R[i]
            n2 = M2 @ r
            nv = np.einsum("abc,b->ca", Mv, r)
            out[0] += n2 / (4 * np.pi * R * R)
            out[1] += n2 / (4 * np.pi * R)
            out[2] += n2
            out[3] += M3 @ r
            out[4:7] += nv / (4 * np.pi * R)
            out[7:10] += nv
        return out.reshape((10,) + tuple(self.shape))


def phi_rosenfeld(n):
    """Rosenfeld FMT Phi (Sec 2.3.1), numpy, complex-safe."""
    n0, n1, n2, n3 = n[0], n[1], n[2], n[3]
    v1 = n[4:7]
    v2 = n[7:10]
    o = 1 - n3
    return (-n0 * np.log(o) + n1 * n2 / o + n2 ** 3 / (24 * np.pi * o ** 2)
            - (v1 * v2).sum(0) / o - n2 * (v2 * v2).sum(0) / (8 * np.pi * o ** 2))


def phi_white_bear(n):
    """White Bear (MFMT) Phi, numpy, complex-safe, closed form in n3 (valid away
    from n3 = 0): the n2^3 term is (n2^3 - 3 n2 v2.v2) phi3(n3) / (36 pi) with
    phi3(x) = [x + (1-x)^2 ln(1-x)] / [x^2 (1-x)^2]."""
    n0, n1, n2, n3 = n[0], n[1], n[2], n[3]
    v1 = n[4:7]
    v2 = n[7:10]
    o = 1 - n3
    phi3 = (n3 + o ** 2 * np.log(o)) / (n3 ** 2 * o ** 2)
    return (-n0 * np.log(o) + (n1 * n2 - (v1 * v2).sum(0)) / o
            + (n2 ** 3 - 3 * n2 * (v2 * v2).sum(0)) * phi3 / (36 * np.pi))
