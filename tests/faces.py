"""Face permeabilities of a cell-permeability problem, formed in NumPy for
the tests (no solver arithmetic beyond the harmonic mean of Sec. 3)."""
import numpy as np


def face_K_from_cells(prob):
    """Face K of a cell-K problem, formed here: the harmonic mean of the two
    cells on an interior face, 2 K_cell on a Dirichlet boundary face (half a
    cell from the centre), 0 on a Neumann face.  Same operation order as the
    cell-K transmissibility, so the two builds agree to the bit."""
    dim = prob.dim
    nx, ny, nz = prob.n3
    K = np.asarray(prob.K, np.float64).reshape(-1, nz, ny, nx)
    comp = [K[a if K.shape[0] > 1 else 0] for a in range(dim)]
    bc = np.asarray(prob.bc)
    nyz, nxz, nxy = ny * nz, nx * nz, nx * ny
    blk = [(bc[:nyz], bc[nyz:2 * nyz]), (bc[2 * nyz:2 * nyz + nxz], bc[2 * nyz + nxz:2 * nyz + 2 * nxz])]
    if dim == 3:
        o = 2 * nyz + 2 * nxz
        blk.append((bc[o:o + nxy], bc[o + nxy:o + 2 * nxy]))
    out = []
    for a in range(dim):
        Kc = comp[a]
        ax = 2 - a  # array axis of grid axis a in (z, y, x) order
        lo = np.take(Kc, range(0, Kc.shape[ax] - 1), axis=ax)
        hi = np.take(Kc, range(1, Kc.shape[ax]), axis=ax)
        s = lo + hi
        inner = np.where(s > 0, (2.0 * lo) * hi / np.where(s > 0, s, 1.0), 0.0)
        first = np.take(Kc, [0], axis=ax)
        last = np.take(Kc, [Kc.shape[ax] - 1], axis=ax)
        shp = list(Kc.shape)
        shp[ax] = 1
        m0 = blk[a][0].reshape(shp).astype(bool)
        m1 = blk[a][1].reshape(shp).astype(bool)
        out.append(np.concatenate([np.where(m0, 2.0 * first, 0.0), inner, np.where(m1, 2.0 * last, 0.0)],
                                  axis=ax).reshape(-1))
    return out
