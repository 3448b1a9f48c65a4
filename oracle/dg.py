"""DG advection operator on a tensor product of two meshes (oracle; test
infrastructure only -- the product path never imports this module).

What is computed (arXiv 2002.08110):

* PDE (Sec. 1.2, Eq. "intro:advection"): df/dt + div(a f) = 0, periodic.
* Weak form per cell in reference coordinates (Sec. 1.3, Eq. "into:adv:ref"):
      (g, |J| df/dt) - (J^{-T} grad_xi g, |J| a f) + <g, |J| n.(a f)*> = 0,
  i.e. M df/dt = A(f) with M the mass matrix.  With the phase-space Jacobian
  J = diag(J_x, J_v) (Sec. 3, first display) the integrand of the cell term is
  grad_xi g . c f with the contravariant speed c = J^{-1} a; on an affine cell
  the face term on the face xi_j = s (s = +-1) is s c_j |J| g f* (Nanson's
  formula n dS = |J| J^{-T} n_hat dS_hat).
* Upwind numerical flux (Sec. 1.3): f* is the trace from the side the flow
  leaves, i.e. from this cell where s c_j > 0, from the neighbour otherwise.
* Element-centric evaluation over all cell pairs (c_x, c_v) (Algorithm 1) and
  the cell operator of Algorithm 2: gather, interpolate to quadrature points,
  multiply by c |J| w, test with the gradient of the basis, add the 2d face
  integrals with the neighbour's trace, apply M^{-1}, scatter.
* Tensor-product quadrature (Sec. 2.5) with n_q = k + 1 Gauss-Legendre points.

Three bases are available (see ``quadrature.Tables1D``): nodal at the
Gauss-Legendre points ("gl", collocation, diagonal M), nodal at the
Gauss-Lobatto points with Gauss quadrature ("gll", the paper's default) and
nodal at the Gauss-Lobatto points with Gauss-Lobatto quadrature ("gllc", the
collocation variant).

Readings taken where the paper is silent:
* the reference cell is [-1, 1]^d;
* the x-mesh is a uniform lattice in coordinates y mapped affinely by x = S y
  (S = identity unless a shear is given); fields and initial data are given as
  functions of the lattice coordinates y, so they stay periodic;
* c_j on a face is the field evaluated at the face quadrature point.

Vector layout (shared with the CUDA library's ABI, a convention, not code):
index = cell * n^d + q, cell = sum_j cc_j * prod_{m<j} N_m over the d cell
coordinates (x dimensions first, x_1 fastest), q = sum_j q_j n^j (x_1 fastest).
"""
import itertools

import numpy as np

from .quadrature import Tables1D


# ---------------------------------------------------------------------------
# velocity fields (Sec. 1.2: a = a(t, x); Sec. 6: a = (v, E(x)))
# ---------------------------------------------------------------------------
class ConstantField:
    """a(y_x, v) = a0, constant and uniform (Sec. 5.1 experiments)."""

    def __init__(self, a):
        self.a = np.asarray(a, dtype=np.float64)

    def __call__(self, yx, v):
        shape = np.broadcast_shapes(yx.shape[:-1], v.shape[:-1])
        return np.broadcast_to(self.a, shape + (len(self.a),)).copy()

    def negated(self):
        return ConstantField(-self.a)


class PhaseSpaceField:
    """a = (v_{1..dx}, E(y_x)): transport in x by the velocity coordinate and
    in v by a field that depends on x only (Sec. 6, the Vlasov field composed
    on the fly).  ``E`` maps lattice x-coordinates (..., dx) to (..., dv).
    ``sign`` = -1 gives the negated field used by the adjoint."""

    def __init__(self, dx, dv, E, sign=1.0):
        if dv < dx:
            raise ValueError("a_x = v[:dx] needs dv >= dx")
        self.dx, self.dv, self.E, self.sign = dx, dv, E, sign

    def __call__(self, yx, v):
        ax = v[..., : self.dx]
        av = np.asarray(self.E(yx), dtype=np.float64)
        shape = np.broadcast_shapes(ax.shape[:-1], av.shape[:-1])
        out = np.concatenate(
            [np.broadcast_to(ax, shape + (self.dx,)), np.broadcast_to(av, shape + (self.dv,))],
            axis=-1,
        )
        return self.sign * out

    def negated(self):
        return PhaseSpaceField(self.dx, self.dv, self.E, -self.sign)


def _axis_apply(M, T, axis):
    """Apply the matrix M along one tensor axis (one factor of a Kronecker product)."""
    return np.moveaxis(np.tensordot(M, T, axes=([1], [axis])), 0, axis)


def _kron_list(mats):
    """Dense Kronecker product acting on column-major (axis 0 fastest) vectors."""
    K = np.ones((1, 1))
    for M in mats:  # axis 0 innermost -> rightmost factor
        K = np.kron(M, K)
    return K


class Problem:
    """Tensor-product mesh T_x (x) T_v with periodic boundaries (Sec. 3.1).

    dx, dv    : dimensions of configuration and velocity space, d = dx + dv
    k         : polynomial degree, n = k + 1 nodes per direction
    cells_x/v : cells per direction
    x_lo/x_hi : lattice box of configuration space; v_lo/v_hi velocity box
    shear     : dx-by-dx matrix S of the affine map x = S y (None: identity)
    deform    : per-direction amplitudes delta of a curved x-mesh (None: affine):
                x_i = y_i + delta_i L_m / (2 pi) sin(2 pi (y_m - lo_m) / L_m),
                m = (i + 1) mod dx, L the box size -- a periodic, non-affine
                deformation of the lattice, so that every quadrature point has
                its own Jacobian (Sec. 5.1 deforms the Cartesian mesh
                slightly for this reason).  Not combined with a shear.
    field     : callable a(y_x, v) -> (..., d) physical velocity
    """

    def __init__(self, dx, dv, k, cells_x, cells_v, x_lo, x_hi, v_lo, v_hi,
                 field, shear=None, basis="gl", deform=None):
        self.dx, self.dv, self.d = dx, dv, dx + dv
        self.k, self.n = k, k + 1
        self.cells = np.array(list(cells_x) + list(cells_v), dtype=np.int64)
        assert len(self.cells) == self.d
        self.lo = np.array(list(x_lo) + list(v_lo), dtype=np.float64)
        self.hi = np.array(list(x_hi) + list(v_hi), dtype=np.float64)
        self.h = (self.hi - self.lo) / self.cells
        self.S = np.eye(dx) if shear is None else np.asarray(shear, dtype=np.float64)
        self.field = field
        self.basis = basis
        self.T = Tables1D(k, basis)
        # Jacobian of the map reference cell -> physical cell, block diagonal
        # (Sec. 3): J_x = S diag(h_x / 2), J_v = diag(h_v / 2).
        J = np.zeros((self.d, self.d))
        J[:dx, :dx] = self.S @ np.diag(self.h[:dx] / 2)
        J[dx:, dx:] = np.diag(self.h[dx:] / 2)
        self.J = J
        self.detJ = float(np.linalg.det(J))
        self.Jinv = np.linalg.inv(J)
        self.deform = None if deform is None else np.asarray(deform, dtype=np.float64)
        if self.deform is not None:
            assert shear is None and basis in ("gl", "gllc")   # diagonal mass only
        self.ncells = int(np.prod(self.cells))
        self.dofs_per_cell = self.n ** self.d
        self.n_dofs = self.ncells * self.dofs_per_cell
        self.strides = np.concatenate([[1], np.cumprod(self.cells)[:-1]]).astype(np.int64)

    # -- bookkeeping -------------------------------------------------------
    def with_field(self, field):
        p = Problem.__new__(Problem)
        p.__dict__.update(self.__dict__)
        p.field = field
        return p

    def cell_coords(self, cell):
        return (cell // self.strides) % self.cells

    def cell_index(self, cc):
        return int(np.sum((np.asarray(cc) % self.cells) * self.strides))

    def neighbour(self, cell, j, s):
        cc = self.cell_coords(cell).copy()
        cc[j] += s
        return self.cell_index(cc)

    def cell_tensor(self, u, cell):
        npc = self.dofs_per_cell
        return np.asarray(u[cell * npc:(cell + 1) * npc], dtype=np.float64).reshape(
            [self.n] * self.d, order="F")

    # -- geometry and field -------------------------------------------------
    def coordinates(self, cell, points):
        """Lattice x-coordinates and velocity coordinates at reference points.

        ``points`` is a list of d 1D arrays (reference coordinates per axis);
        returns (yx, v) on the tensor grid, shapes (..., dx) and (..., dv)."""
        cc = self.cell_coords(cell)
        axes = [self.lo[j] + self.h[j] * (cc[j] + (np.asarray(points[j]) + 1.0) / 2.0)
                for j in range(self.d)]
        grid = np.meshgrid(*axes, indexing="ij")
        Y = np.stack(grid, axis=-1)
        return Y[..., : self.dx], Y[..., self.dx:]

    def node_coordinates(self, cell):
        return self.coordinates(cell, [self.T.nodes] * self.d)

    def physical_x(self, yx):
        """x = Phi(y) of the curved mesh (the identity map S y otherwise)."""
        if self.deform is None:
            return yx @ self.S.T
        L = self.hi[:self.dx] - self.lo[:self.dx]
        x = np.array(yx, dtype=np.float64, copy=True)
        for i in range(self.dx):
            m = (i + 1) % self.dx
            x[..., i] += self.deform[i] * L[m] / (2 * np.pi) * np.sin(
                2 * np.pi * (yx[..., m] - self.lo[m]) / L[m])
        return x

    def jacobian(self, cell, points):
        """(J, |J|) at the given reference points: J has shape (..., d, d).
        For the curved mesh J_x = (dPhi/dy) diag(h_x / 2) at every point."""
        yx, v = self.coordinates(cell, points)
        shape = yx.shape[:-1]
        if self.deform is None:
            J = np.broadcast_to(self.J, shape + (self.d, self.d))
            return J, np.full(shape, self.detJ)
        dx = self.dx
        L = self.hi[:dx] - self.lo[:dx]
        DPhi = np.broadcast_to(np.eye(dx), shape + (dx, dx)).copy()
        for i in range(dx):
            m = (i + 1) % dx
            DPhi[..., i, m] += self.deform[i] * np.cos(2 * np.pi * (yx[..., m] - self.lo[m]) / L[m])
        J = np.zeros(shape + (self.d, self.d))
        J[..., :dx, :dx] = DPhi * (self.h[:dx] / 2)
        J[..., dx:, dx:] = np.diag(self.h[dx:] / 2)
        return J, np.linalg.det(J)

    def contravariant_speed(self, cell, points):
        """c = J^{-1} a at the given reference points, shape (..., d)."""
        yx, v = self.coordinates(cell, points)
        a = self.field(yx, v)
        if self.deform is None:
            return a @ self.Jinv.T
        J, _ = self.jacobian(cell, points)
        return np.linalg.solve(J, a[..., None])[..., 0]

    def _detJ(self, cell, points):
        """|J| at the points (a scalar for the affine mesh)."""
        if self.deform is None:
            return self.detJ
        return self.jacobian(cell, points)[1]

    def interpolate(self, f, cell_list=None):
        """Nodal interpolation of f(y_x, v) (the initial state)."""
        cells = range(self.ncells) if cell_list is None else cell_list
        out = []
        for e in cells:
            yx, v = self.node_coordinates(e)
            out.append(np.asarray(f(yx, v), dtype=np.float64).reshape(-1, order="F"))
        return np.concatenate(out)

    # -- the operator, axis by axis ------------------------------------------
    def _face_trace(self, U, j, l):
        """Interpolate the cell tensor U to the quadrature points of the face
        normal to axis j (l = basis values at the face coordinate); axis j
        keeps length 1."""
        T = self.T
        G = _axis_apply(l[None, :], U, j)
        for m in range(self.d):
            if m != j:
                G = _axis_apply(T.B, G, m)
        return G

    def cell_residual(self, u, cell, absolute=False):
        """b = A(u) restricted to the test functions of ``cell`` (before M^{-1}).

        absolute=True evaluates the same sums with the absolute value of every
        factor and term (the "term scale" |A| |u| against which the rounding
        error of a reduced-precision evaluation is measured)."""
        T, d = self.T, self.d
        if absolute:
            return self._cell_residual_abs(u, cell)
        Ue = self.cell_tensor(u, cell)
        # step 2: interpolate to quadrature points
        Uq = Ue
        for m in range(d):
            Uq = _axis_apply(T.B, Uq, m)
        C = self.contravariant_speed(cell, [T.zeta] * d)
        W = _outer_weights([T.w] * d)
        dJ = self._detJ(cell, [T.zeta] * d)
        b = np.zeros_like(Ue)
        for j in range(d):
            F = W * dJ * C[..., j] * Uq
            G = F
            for m in range(d):
                G = _axis_apply((T.Bd if m == j else T.B).T, G, m)
            b += G
        # step 3: faces
        for j in range(d):
            for s in (1, -1):
                ls, lo = (T.lp, T.lm) if s > 0 else (T.lm, T.lp)
                own = self._face_trace(Ue, j, ls)
                nb = self._face_trace(self.cell_tensor(u, self.neighbour(cell, j, s)), j, lo)
                pts = [T.zeta] * d
                pts[j] = np.array([float(s)])
                cj = self.contravariant_speed(cell, pts)[..., j]
                ustar = np.where(s * cj > 0, own, nb)
                wf = [T.w] * d
                wf[j] = np.array([1.0])
                flux = _outer_weights(wf) * self._detJ(cell, pts) * cj * ustar
                G = flux
                for m in range(d):
                    if m != j:
                        G = _axis_apply(T.B.T, G, m)
                G = _axis_apply(ls[:, None], G, j)
                b -= s * G
        return b

    def _cell_residual_abs(self, u, cell):
        T, d = self.T, self.d
        aB, aBd = np.abs(T.B), np.abs(T.Bd)
        Ue = np.abs(self.cell_tensor(u, cell))
        Uq = Ue
        for m in range(d):
            Uq = _axis_apply(aB, Uq, m)
        C = np.abs(self.contravariant_speed(cell, [T.zeta] * d))
        W = _outer_weights([T.w] * d)
        dJ = self._detJ(cell, [T.zeta] * d)
        b = np.zeros_like(Ue)
        for j in range(d):
            G = W * dJ * C[..., j] * Uq
            for m in range(d):
                G = _axis_apply((aBd if m == j else aB).T, G, m)
            b += G
        for j in range(d):
            for s in (1, -1):
                ls, lo = (T.lp, T.lm) if s > 0 else (T.lm, T.lp)
                own = self._face_trace_abs(Ue, j, np.abs(ls))
                nbu = np.abs(self.cell_tensor(u, self.neighbour(cell, j, s)))
                nb = self._face_trace_abs(nbu, j, np.abs(lo))
                pts = [T.zeta] * d
                pts[j] = np.array([float(s)])
                cj = self.contravariant_speed(cell, pts)[..., j]
                ustar = np.where(s * cj > 0, own, nb)
                wf = [T.w] * d
                wf[j] = np.array([1.0])
                G = _outer_weights(wf) * self._detJ(cell, pts) * np.abs(cj) * ustar
                for m in range(d):
                    if m != j:
                        G = _axis_apply(aB.T, G, m)
                G = _axis_apply(np.abs(ls)[:, None], G, j)
                b += G
        return b

    def _face_trace_abs(self, U, j, l):
        G = _axis_apply(l[None, :], U, j)
        for m in range(self.d):
            if m != j:
                G = _axis_apply(np.abs(self.T.B), G, m)
        return G

    def apply_abs(self, u, cells=None):
        """Term scale |M^{-1}| |A| |u| (collocation basis: M^{-1} diagonal)."""
        assert self.basis in ("gl", "gllc")   # collocation: diagonal mass
        u = np.asarray(u, dtype=np.float64)
        sel = range(self.ncells) if cells is None else cells
        out = [self.apply_mass_inverse(self._cell_residual_abs(u, e), e).reshape(-1, order="F")
               for e in sel]
        return np.concatenate(out) if cells is None else np.stack(out)

    def mass_1d(self):
        T = self.T
        return T.B.T @ np.diag(T.w) @ T.B

    def apply_mass_inverse(self, b, cell=None):
        """M^{-1} b on one cell (``cell`` is needed on the curved mesh, where
        the collocation mass is diag(W |J(q)|))."""
        if self.deform is not None:
            W = _outer_weights([self.T.w] * self.d)
            return b / (W * self._detJ(cell, [self.T.zeta] * self.d))
        M1 = self.mass_1d()
        y = b / self.detJ
        for m in range(self.d):
            y = _axis_apply(np.linalg.inv(M1), y, m)
        return y

    def apply_mass(self, y, cell=None):
        if self.deform is not None:
            W = _outer_weights([self.T.w] * self.d)
            return y * W * self._detJ(cell, [self.T.zeta] * self.d)
        M1 = self.mass_1d()
        b = y * self.detJ
        for m in range(self.d):
            b = _axis_apply(M1, b, m)
        return b

    def apply(self, u, cells=None):
        """du = M^{-1} A(u) for all cells (flat vector) or for a list of cells
        (returns an array of shape (len(cells), n^d))."""
        u = np.asarray(u, dtype=np.float64)
        assert u.shape == (self.n_dofs,)
        sel = range(self.ncells) if cells is None else cells
        out = [self.apply_mass_inverse(self.cell_residual(u, e), e).reshape(-1, order="F")
               for e in sel]
        return np.concatenate(out) if cells is None else np.stack(out)

    def apply_adjoint(self, y, cells=None):
        """L^T y by the dense cell blocks (brute force: sums the transposed
        row blocks of every cell that couples to the requested cells)."""
        y = np.asarray(y, dtype=np.float64)
        sel = range(self.ncells) if cells is None else list(cells)
        out = []
        for e in sel:
            acc = np.zeros(self.dofs_per_cell)
            rows = {e}
            for j in range(self.d):
                for s in (1, -1):
                    rows.add(self.neighbour(e, j, s))
            for r in rows:
                blocks = self.dense_cell_blocks(r)
                if e in blocks:
                    npc = self.dofs_per_cell
                    acc += blocks[e].T @ y[r * npc:(r + 1) * npc]
            out.append(acc)
        return np.concatenate(out) if cells is None else np.stack(out)

    # -- the same operator as dense Kronecker matrices (tiny cells) -----------
    def dense_cell_blocks(self, cell):
        """Row blocks of L = M^{-1} A for one cell as dense matrices:
        {column cell: n^d x n^d block}.  Built from explicit Kronecker products
        of the 1D tables (brute force route)."""
        T, d, n = self.T, self.d, self.n
        if n ** d > 1296:
            raise ValueError("dense blocks only for small cells")
        KB = _kron_list([T.B] * d)
        W = _outer_weights([T.w] * d).reshape(-1, order="F")
        C = self.contravariant_speed(cell, [T.zeta] * d)
        Cf = C.reshape(-1, d, order="F")
        dJ = np.broadcast_to(self._detJ(cell, [T.zeta] * d), [n] * d).reshape(-1, order="F")
        A_own = np.zeros((n ** d, n ** d))
        blocks = {}
        for j in range(d):
            KBd = _kron_list([T.Bd if m == j else T.B for m in range(d)])
            A_own += KBd.T @ np.diag(W * dJ * Cf[:, j]) @ KB
        for j in range(d):
            for s in (1, -1):
                ls, lo = (T.lp, T.lm) if s > 0 else (T.lm, T.lp)
                Ts = _kron_list([ls[None, :] if m == j else T.B for m in range(d)])
                Tn = _kron_list([lo[None, :] if m == j else T.B for m in range(d)])
                pts = [T.zeta] * d
                pts[j] = np.array([float(s)])
                cj = self.contravariant_speed(cell, pts)[..., j].reshape(-1, order="F")
                wf = [T.w] * d
                wf[j] = np.array([1.0])
                Wf = _outer_weights(wf).reshape(-1, order="F")
                out = (s * cj > 0).astype(np.float64)
                dJf = self._detJ(cell, pts)
                dJf = np.asarray(dJf).reshape(-1, order="F") if np.ndim(dJf) else dJf
                A_own += -s * Ts.T @ np.diag(Wf * dJf * cj * out) @ Ts
                nbc = self.neighbour(cell, j, s)
                blk = -s * Ts.T @ np.diag(Wf * dJf * cj * (1.0 - out)) @ Tn
                blocks[nbc] = blocks.get(nbc, 0.0) + blk
        blocks[cell] = blocks.get(cell, 0.0) + A_own
        M = KB.T @ np.diag(W * dJ) @ KB
        Minv = np.linalg.inv(M)
        return {c: Minv @ B for c, B in blocks.items()}

    def apply_dense(self, u):
        u = np.asarray(u, dtype=np.float64)
        npc = self.dofs_per_cell
        out = np.zeros(self.n_dofs)
        for e in range(self.ncells):
            for c, B in self.dense_cell_blocks(e).items():
                out[e * npc:(e + 1) * npc] += B @ u[c * npc:(c + 1) * npc]
        return out

    def assemble(self):
        """Global sparse L = M^{-1} A (scipy.sparse CSR) from the dense blocks."""
        import scipy.sparse as sp
        npc = self.dofs_per_cell
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(npc), np.arange(npc), indexing="ij")
        for e in range(self.ncells):
            for c, B in self.dense_cell_blocks(e).items():
                rows.append((e * npc + ii).ravel())
                cols.append((c * npc + jj).ravel())
                vals.append(B.ravel())
        L = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n_dofs, self.n_dofs))
        return L.tocsr()

    def mass_diagonal(self):
        """Diagonal of M for the collocation basis (|J| times the weights)."""
        assert self.basis in ("gl", "gllc")   # collocation: diagonal mass
        W = _outer_weights([self.T.w] * self.d).reshape(-1, order="F")
        if self.deform is None:
            return np.tile(W * self.detJ, self.ncells)
        pts = [self.T.zeta] * self.d
        return np.concatenate([W * np.asarray(self._detJ(e, pts)).reshape(-1, order="F")
                               for e in range(self.ncells)])

    # -- Vlasov-Poisson coupling (Sec. 6) -------------------------------------
    def charge_density(self, u, x_cells=None):
        """rho(x_q) = 1 - int f(x_q, v) dv at every x node, from the definition:
        the v integral by the cell quadrature of the v mesh (|J_v| times the
        product of the 1D weights), collocation basis.  Returns an array of
        shape (x cells, x nodes) with x cells and nodes lexicographic (only
        the rows of ``x_cells`` if given)."""
        assert self.basis in ("gl", "gllc")   # collocation: diagonal mass
        dx, dv, n = self.dx, self.dv, self.n
        ncx = int(np.prod(self.cells[:dx]))
        ncv = int(np.prod(self.cells[dx:]))
        detJv = float(np.prod(self.h[dx:] / 2))
        Wv = _outer_weights([self.T.w] * dv).reshape(-1, order="F")
        rows = range(ncx) if x_cells is None else list(x_cells)
        rho = np.ones((len(rows), n ** dx))
        for r, cx in enumerate(rows):
            for cv in range(ncv):
                e = cx + ncx * cv
                f = self.cell_tensor(u, e).reshape(n ** dx, n ** dv, order="F")
                rho[r] -= detJv * (f @ Wv)
        return rho

    # -- integrals -----------------------------------------------------------
    def integrals(self, u):
        """(int u, int u^2, max |u| at nodes) with the cell quadrature."""
        u = np.asarray(u, dtype=np.float64)
        T = self.T
        W = _outer_weights([T.w] * self.d)
        mass = l2 = 0.0
        for e in range(self.ncells):
            Uq = self.cell_tensor(u, e)
            for m in range(self.d):
                Uq = _axis_apply(T.B, Uq, m)
            dJ = self._detJ(e, [T.zeta] * self.d)
            mass += float(np.sum(W * dJ * Uq))
            l2 += float(np.sum(W * dJ * Uq * Uq))
        return mass, l2, float(np.max(np.abs(u)))


def _outer_weights(ws):
    W = np.ones([len(w) for w in ws])
    for j, w in enumerate(ws):
        shape = [1] * len(ws)
        shape[j] = len(w)
        W = W * np.asarray(w).reshape(shape)
    return W
