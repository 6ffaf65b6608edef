"""Brute-force FP64 gradient oracle for the filtered LB-MHD step.

TEST INFRASTRUCTURE ONLY (used by tests/ to check the CUDA adjoint).  The
step is written again from the paper with plain PyTorch CPU tensor ops in
float64, and PyTorch's tape (autograd) differentiates it: no hand-written
derivative anywhere.  It shares no code with the CUDA path or with
lbmhd_oracle.c; a CPU test pins its forward to the C oracle.

Method (Sec. 1.2 streaming, Sec. 3 MRT / SRT collisions, the local
Smagorinsky rates of the reading in lbmhd_oracle.c):
  stream: f_i(x) <- f_i(x - c_i), g_k(x) <- g_k(x - C_k) (periodic roll)
  moments: rho, rho u, B;  M = T f with T from Eq. FluidTMatrix
  equilibria of Eq. KinMomentEq; n = M - M^eq
  tau_e = (tau_nu + sqrt(tau_nu^2 + 18 C_S Delta^2 Q / rho)) / 2,
  Q = sqrt(n_4^2 + 4 n_3^2);  tau_m likewise from J (magnetic current)
  relax in moment space, back with T^-1;  g <- g - (g - g^eq) / tau_m
At Q = 0 or J = 0 (non-differentiable points) the derivative is taken as
0, as the CUDA adjoint does.
"""
from __future__ import annotations

import torch

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
MCX = [0, 1, 0, -1, 0]
MCY = [0, 0, 1, 0, -1]
W9 = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
W5 = [1 / 3] + [1 / 6] * 4


def tmatrix() -> torch.Tensor:
    rows = []
    for i in range(9):
        cx, cy = CX[i], CY[i]
        rows.append([1, cx, cy, cx * cy, cx * cx - cy * cy, 3 * cx * cy * cy - 2 * cx,
                     3 * cy * cx * cx - 2 * cy, 4 - 9 * (cx * cx + cy * cy - 2 * cx * cx * cy * cy),
                     4 - 4 * (cx * cx + cy * cy) + 3 * cx * cx * cy * cy])
    return torch.tensor(rows, dtype=torch.float64).T  # T[j, i]


class _SafeSqrt(torch.autograd.Function):
    """sqrt with derivative 0 at 0 (subgradient choice at the kink)."""

    @staticmethod
    def forward(ctx, x):
        y = torch.sqrt(x)
        ctx.save_for_backward(y)
        return y

    @staticmethod
    def backward(ctx, gy):
        (y,) = ctx.saved_tensors
        return torch.where(y > 0, gy / (2 * torch.where(y > 0, y, torch.ones_like(y))),
                           torch.zeros_like(y))


def equilibrium(rho, ux, uy, bx, by):
    """f^eq (9, ny, nx) and g^eq (10, ny, nx) of Sec. 3."""
    u2 = ux * ux + uy * uy
    b2 = bx * bx + by * by
    f = []
    for i in range(9):
        cu = CX[i] * ux + CY[i] * uy
        cb = CX[i] * bx + CY[i] * by
        c2 = CX[i] ** 2 + CY[i] ** 2
        f.append(W9[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u2)
                 + 4.5 * W9[i] * (0.5 * b2 * c2 - cb * cb))
    g = []
    for k in range(5):
        Cu = MCX[k] * ux + MCY[k] * uy
        CB = MCX[k] * bx + MCY[k] * by
        g.append(W5[k] * (bx + 3 * (Cu * bx - CB * ux)))
        g.append(W5[k] * (by + 3 * (Cu * by - CB * uy)))
    return torch.stack(f), torch.stack(g)


def stream(st):
    out = []
    for p in range(19):
        if p < 9:
            cx, cy = CX[p], CY[p]
        else:
            cx, cy = MCX[(p - 9) // 2], MCY[(p - 9) // 2]
        out.append(torch.roll(st[p], shifts=(cy, cx), dims=(0, 1)))
    return torch.stack(out)


def collide(z, tau_nu, tau_eta, C_S, delta=1.0, rates=(0.0, 0.0, 0.0, 0.0), les=True):
    T = tmatrix()
    f, g = z[:9], z[9:]
    rho = f.sum(0)
    jx = sum(CX[i] * f[i] for i in range(9))
    jy = sum(CY[i] * f[i] for i in range(9))
    ux, uy = jx / rho, jy / rho
    bx = g[0::2].sum(0)
    by = g[1::2].sum(0)
    M = torch.einsum("ji,iyx->jyx", T, f)
    j2 = jx * jx + jy * jy
    Meq = torch.stack([rho, jx, jy, jx * jy / rho - bx * by,
                       (jx * jx - jy * jy) / rho - bx * bx + by * by, -jx, -jy, -3 * j2 / rho,
                       5.0 / 3.0 * rho - 3 * j2 / rho])
    n = M - Meq
    if les:
        Q = _SafeSqrt.apply(n[4] * n[4] + 4 * n[3] * n[3])
        tau_e = 0.5 * (tau_nu + torch.sqrt(tau_nu * tau_nu + 18 * C_S * delta * delta * Q / rho))
        Ny1 = sum(MCX[k] * g[2 * k + 1] for k in range(5))
        Nx2 = sum(MCY[k] * g[2 * k] for k in range(5))
        E = ux * by - uy * bx
        J = torch.abs((Ny1 - E) - (Nx2 + E))
        tau_m = 0.5 * (tau_eta + torch.sqrt(tau_eta * tau_eta + 36 * C_S * delta * delta * J))
    else:
        tau_e = tau_nu * torch.ones_like(rho)
        tau_m = tau_eta * torch.ones_like(rho)
    s_nu = 1.0 / tau_e
    s5, s6, s7, s8 = rates
    zero = torch.zeros_like(rho)
    s = torch.stack([zero, zero, zero, s_nu, s_nu,
                     s5 * torch.ones_like(rho) if s5 > 0 else (1.0 / tau_nu) * torch.ones_like(rho),
                     s6 * torch.ones_like(rho) if s6 > 0 else (1.0 / tau_nu) * torch.ones_like(rho),
                     s7 * torch.ones_like(rho) if s7 > 0 else s_nu,
                     s8 * torch.ones_like(rho) if s8 > 0 else s_nu])
    Ms = M - s * n
    norm2 = (T * T).sum(1)
    fs = torch.einsum("ji,jyx->iyx", T, Ms / norm2[:, None, None])
    _, geq = equilibrium(rho, ux, uy, bx, by)
    gs = g - (g - geq) / tau_m
    return torch.cat([fs, gs])


def rollout(rho0, ux0, uy0, bx0, by0, tau_nu, tau_eta, C_S, nsteps, delta=1.0,
            rates=(0.0, 0.0, 0.0, 0.0), les=True):
    """Final moments (rho, ux, uy, bx, by) after nsteps from the equilibrium
    state of the given fields; every input may require grad."""
    f, g = equilibrium(rho0, ux0, uy0, bx0, by0)
    st = torch.cat([f, g])
    for _ in range(nsteps):
        st = collide(stream(st), tau_nu, tau_eta, C_S, delta, rates, les)
    f, g = st[:9], st[9:]
    rho = f.sum(0)
    ux = sum(CX[i] * f[i] for i in range(9)) / rho
    uy = sum(CY[i] * f[i] for i in range(9)) / rho
    return rho, ux, uy, g[0::2].sum(0), g[1::2].sum(0)


def gradients(fields, tau_nu, tau_eta, C_S, nsteps, weights, **kw):
    """d/d(inputs) of sum_k <weights_k, output_k> by the tape.  Returns
    (value, dict of gradients: rho0, ux0, uy0, bx0, by0, tau_nu, tau_eta, C_S)."""
    leaves = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in fields]
    th = [torch.tensor(float(v), dtype=torch.float64, requires_grad=True)
          for v in (tau_nu, tau_eta, C_S)]
    out = rollout(*leaves, th[0], th[1], th[2], nsteps, **kw)
    val = sum((o * torch.as_tensor(w, dtype=torch.float64)).sum() for o, w in zip(out, weights))
    val.backward()
    names = ["rho0", "ux0", "uy0", "bx0", "by0"]
    grads = {n: l.grad.numpy() for n, l in zip(names, leaves)}
    grads.update(tau_nu=float(th[0].grad), tau_eta=float(th[1].grad), C_S=float(th[2].grad))
    return val.item(), grads
