"""FP64 reference of the quasi-neutral hybrid model -- TEST INFRASTRUCTURE ONLY (see the package
docstring).

The paper's analytic model (Eqs. 1-6), as a simulation: a kinetic electron beam in the transverse
plane, the plasma return current as a fluid, and the axial vector potential from Ampere's law
without the displacement current.  Units: time 1/w_p, length c/w_p, velocity c, a = e A_z /(m c^2)
(electron charge -e), densities n0.  With the paper's sign conventions the equations read

  Ampere (Eq. 2):           lap a = n_b beta_bz + n_p beta_p           (beam and plasma currents)
  plasma flow (Eq. 3):      d beta_p / dt + nu beta_p = d a / dt
  beam, transverse (Eq. 4): d u_perp / dt = -(beta_z - beta_p) grad a  (u = gamma beta)
  beam, axial (Eq. 6):      u_z = P + a,  P constant per particle (canonical momentum)

Dropping the displacement current keeps the plasma quasi-neutral, so the plasma density that
carries the return current is the local n_p = n0 - n_b (the remark after Eq. 7 on the actual
plasma density).  With it the total energy of Eq. 7 -- beam energy, magnetic energy and the plasma
kinetic energy sum n_p beta_p^2 / 2 -- is an exact invariant of the collisionless model; the
paper's form (its terms 2 and 4) is this one with beta_p = a.

Discretisation (a reading; the paper gives none): periodic nx x ny grid, a and beta_p at the
nodes, the 5-point Laplacian; beam particles at cell coordinates X = x/dx; bilinear (CIC)
interpolation of a and beta_p and the gradient of the bilinear interpolant of a; CIC deposit of
the beam density w and current w beta_z; n_p = max(n0 - n_b, 0) per node.  One step n -> n+1:

  1. at X^n: a, grad a, beta_p;  u_z = P + a;  gamma = sqrt(1 + |u_perp^{n-1/2}|^2 + u_z^2)
  2. u_perp^{n+1/2} = u_perp^{n-1/2} - dt (u_z / gamma - beta_p) grad a
  3. X^{n+1} = X^n + dt u_perp^{n+1/2} / (gamma' dx),  gamma' from u_perp^{n+1/2} and u_z
  4. beam density and current at X^{n+1}, with u_z* = P + a^n(X^{n+1})
  5. (lap - n_p) a^{n+1} = n_b beta_b + n_p (beta_p^n - a^n - nu dt beta_p^n)   (sparse direct solve)
  6. beta_p^{n+1} = beta_p^n + a^{n+1} - a^n - nu dt beta_p^n

Diagnostics: magnetic energy sum((D+ a)^2)/2 dx dy (B_perp = -e_z x grad a; D+ the forward
differences whose product gives the 5-point Laplacian), beam energy sum w (gamma - 1) dx dy,
plasma energy sum n_p beta_p^2 / 2 dx dy with n_p from the beam's current positions.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def laplacian_eigenvalues(nx, ny, dx, dy):
    """Eigenvalues of the periodic 5-point Laplacian on the FFT modes, shape (ny, nx)."""
    lx = -(4.0 / dx ** 2) * np.sin(np.pi * np.arange(nx) / nx) ** 2
    ly = -(4.0 / dy ** 2) * np.sin(np.pi * np.arange(ny) / ny) ** 2
    return ly[:, None] + lx[None, :]


def screened_solve(S, n_p, dx, dy):
    """a with (lap - n_p) a = S on the periodic grid (numpy FFT)."""
    ny, nx = S.shape
    lam = laplacian_eigenvalues(nx, ny, dx, dy) - n_p
    return np.real(np.fft.ifft2(np.fft.fft2(S) / lam))


def laplacian_matrix(nx, ny, dx, dy):
    """The periodic 5-point Laplacian as a sparse (ny nx) x (ny nx) matrix, node (j, i) at j nx + i."""
    def ring(n, h):
        d = sp.diags([np.full(n, -2.0), np.ones(n - 1), np.ones(n - 1)], [0, -1, 1], format="lil")
        d[0, n - 1] += 1.0
        d[n - 1, 0] += 1.0
        return d.tocsr() / h ** 2
    return (sp.kron(sp.identity(ny), ring(nx, dx)) + sp.kron(ring(ny, dy), sp.identity(nx))).tocsc()


def quasineutral_solve(S, n_p, dx, dy):
    """a with (lap - diag n_p) a = S on the periodic grid, n_p a per-node field (sparse LU)."""
    ny, nx = S.shape
    A = laplacian_matrix(nx, ny, dx, dy) - sp.diags(np.asarray(n_p, np.float64).reshape(-1))
    return spla.spsolve(A.tocsc(), S.reshape(-1)).reshape(ny, nx)


def linear_growth_rate(k, beta0, gamma0, n_b, n0=1.0):
    """Growth rate of a small transverse filamentation mode k of a cold beam in this model with
    the return current initially neutralising (beta_p0 = -n_b beta0 / n_p, n_p = n0 - n_b), nu = 0:
    Gamma^2 = beta0^2 n_b k^2 (n0 / n_p)^2 / (gamma0 (k^2 + n_p + n_b / gamma0^3)).
    Linearising Eqs. 2-4 and 6 about that state: delta u_z = delta a (so delta beta_z =
    delta a / gamma0^3), the plasma current changes by n_p delta a - beta_p0 delta n_b, hence
    delta a = -beta0 (n0 / n_p) delta n_b / (k^2 + n_p + n_b / gamma0^3); the displacement xi obeys
    gamma0 xi'' = -(beta0 - beta_p0) d(delta a)/dx with beta0 - beta_p0 = beta0 n0 / n_p and
    delta n_b = -n_b dxi/dx.  Without the beta_p0 terms (the paper's beta0 ~ v_bz / c) and with
    gamma0 = 1 this is the collisionless cold limit of Eq. 11."""
    n_p = n0 - n_b
    return np.sqrt(beta0 ** 2 * n_b * k ** 2 * (n0 / n_p) ** 2
                   / (gamma0 * (k ** 2 + n_p + n_b / gamma0 ** 3)))


class HybridSim:
    def __init__(self, nx, ny, dx, dy, dt, n0, nu, w):
        self.nx, self.ny, self.dx, self.dy, self.dt = nx, ny, dx, dy, dt
        self.n0, self.nu, self.w = float(n0), float(nu), float(w)
        self.a = np.zeros((ny, nx))
        self.beta_p = np.zeros((ny, nx))
        self.X = self.Y = self.ux = self.uy = self.P = np.zeros(0)
        self.step_index = 0

    def load(self, X, Y, ux, uy, uz, beta_p):
        """Beam particles (cell coordinates, momenta) with a = 0, and the plasma velocity field."""
        self.X = np.asarray(X, np.float64).copy()
        self.Y = np.asarray(Y, np.float64).copy()
        self.ux = np.asarray(ux, np.float64).copy()
        self.uy = np.asarray(uy, np.float64).copy()
        self.P = np.asarray(uz, np.float64).copy() - self._interp(self.a, self.X, self.Y)
        self.beta_p = np.broadcast_to(np.asarray(beta_p, np.float64), (self.ny, self.nx)).copy()

    # -- interpolation and deposit (CIC)
    def _cic(self, X, Y):
        i = np.floor(X).astype(np.int64)
        j = np.floor(Y).astype(np.int64)
        fx, fy = X - i, Y - j
        return i % self.nx, j % self.ny, (i + 1) % self.nx, (j + 1) % self.ny, fx, fy

    def _interp(self, F, X, Y):
        i0, j0, i1, j1, fx, fy = self._cic(X, Y)
        return ((1 - fx) * (1 - fy) * F[j0, i0] + fx * (1 - fy) * F[j0, i1]
                + (1 - fx) * fy * F[j1, i0] + fx * fy * F[j1, i1])

    def _grad(self, F, X, Y):
        i0, j0, i1, j1, fx, fy = self._cic(X, Y)
        gx = ((1 - fy) * (F[j0, i1] - F[j0, i0]) + fy * (F[j1, i1] - F[j1, i0])) / self.dx
        gy = ((1 - fx) * (F[j1, i0] - F[j0, i0]) + fx * (F[j1, i1] - F[j0, i1])) / self.dy
        return gx, gy

    def _deposit(self, X, Y, q):
        i0, j0, i1, j1, fx, fy = self._cic(X, Y)
        out = np.zeros(self.nx * self.ny)
        for ii, jj, wgt in ((i0, j0, (1 - fx) * (1 - fy)), (i1, j0, fx * (1 - fy)),
                            (i0, j1, (1 - fx) * fy), (i1, j1, fx * fy)):
            out += np.bincount(jj * self.nx + ii, weights=q * wgt, minlength=self.nx * self.ny)
        return out.reshape(self.ny, self.nx)

    def push(self, X, Y, ux, uy, P):
        """Steps 1-3 for the given particles in the current fields: (X, Y, ux, uy) after the move."""
        a, bp, dt = self.a, self.beta_p, self.dt
        ua = self._interp(a, X, Y)
        gx, gy = self._grad(a, X, Y)
        bpp = self._interp(bp, X, Y)
        uz = P + ua
        g = np.sqrt(1.0 + ux ** 2 + uy ** 2 + uz ** 2)
        f = uz / g - bpp
        ux = ux - dt * f * gx
        uy = uy - dt * f * gy
        g2 = np.sqrt(1.0 + ux ** 2 + uy ** 2 + uz ** 2)
        X = (X + dt * ux / (g2 * self.dx)) % self.nx
        Y = (Y + dt * uy / (g2 * self.dy)) % self.ny
        return X, Y, ux, uy

    def step(self, n=1):
        for _ in range(n):
            a, bp, dt = self.a, self.beta_p, self.dt
            self.X, self.Y, self.ux, self.uy = self.push(self.X, self.Y, self.ux, self.uy, self.P)
            uzs = self.P + self._interp(a, self.X, self.Y)
            gs = np.sqrt(1.0 + self.ux ** 2 + self.uy ** 2 + uzs ** 2)
            jb = self._deposit(self.X, self.Y, self.w * uzs / gs)
            n_p = self.plasma_density()
            rhs = jb + n_p * (bp - a - self.nu * dt * bp)
            a_new = quasineutral_solve(rhs, n_p, self.dx, self.dy)
            self.beta_p = bp + a_new - a - self.nu * dt * bp
            self.a = a_new
            self.step_index += 1

    def plasma_density(self):
        """n_p = max(n0 - n_b, 0) per node, n_b the CIC beam density at the current positions."""
        nb = self._deposit(self.X, self.Y, np.full(self.X.shape[0], self.w))
        return np.maximum(self.n0 - nb, 0.0)

    def energies(self):
        """(magnetic, beam kinetic, plasma kinetic), each integrated over the plane."""
        dA = self.dx * self.dy
        dxa = (np.roll(self.a, -1, axis=1) - self.a) / self.dx
        dya = (np.roll(self.a, -1, axis=0) - self.a) / self.dy
        uz = self.P + self._interp(self.a, self.X, self.Y)
        g = np.sqrt(1.0 + self.ux ** 2 + self.uy ** 2 + uz ** 2)
        return (0.5 * np.sum(dxa ** 2 + dya ** 2) * dA, self.w * np.sum(g - 1.0) * dA,
                0.5 * np.sum(self.plasma_density() * self.beta_p ** 2) * dA)
