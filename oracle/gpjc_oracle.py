"""FP64 CPU oracle for group-patch joint compression (arXiv 2601.05418).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
baseline of the benchmark may import this module; the product path never
does.  It shares no code with the CUDA library: plain numpy in float64 /
complex128, with numpy's FFT, matmul and Hermitian eigensolver as library
steps, written to be checked against the paper by eye.

Notation follows the paper: N_C coils, N_tx oversampled readout samples,
patch of w samples, N_s = N_C * w, N_s' = keep, group g, A_g (Eq. 12),
P_g (Eq. 7-11), S' = A_g S_g (Eq. 13), E' = A_g E_g (Eq. 14-15).

Index conventions (readings of the paper recorded in the design notes):
  * centred indices x_c = x - N_x/2, t_c = t - N_tx/2, ky_c = ky - N_y/2 ...
  * readout encoding exp(-i 2 pi t_c x_c / N_tx) / sqrt(N_tx)  (Eq. 1, 4)
  * wave phase phi(t,y,z) = 2 pi [a_y(t) y_c/N_y + a_z(t) z_c/N_z],
    a_y = kappa_y (1 - cos th)/2, a_z = kappa_z sin(th)/2,
    th = 2 pi cycles t / N_tx                                   (Eq. 3)
  * patch vector index i = n * w + tau (coil-major)
  * raw data layout S[line][coil][t]; compressed S'[line][off_p + k]
"""
from __future__ import annotations

import math
from typing import Callable, Dict, Optional, Tuple

import numpy as np

PI = math.pi


# ============================================================ bookkeeping ==

def patch_offsets(patch_group: np.ndarray, keep: np.ndarray) -> np.ndarray:
    """off[p] = sum_{q<p} keep[g(q)] (position of patch p in the compressed
    readout; Eq. 15 with N'_tx = sum_p keep[g(p)])."""
    off = np.zeros(len(patch_group), np.int64)
    acc = 0
    for p, g in enumerate(patch_group):
        off[p] = acc
        acc += int(keep[g])
    return off


def ntx_compressed(patch_group: np.ndarray, keep: np.ndarray) -> int:
    """N'_tx = sum over patches of the kept dimension of the patch's group."""
    return int(sum(int(keep[g]) for g in patch_group))


def reference_patch(patch_group: np.ndarray, n_groups: int) -> np.ndarray:
    """p_g: the first patch carrying group g (its encoding defines P_g)."""
    ref = np.full(n_groups, -1, np.int64)
    for p, g in enumerate(patch_group):
        if ref[g] < 0:
            ref[g] = p
    return ref


def periodic_grouping_ok(patch_group, w: int, period: int) -> bool:
    """Same-group patches must start a whole number of modulation periods
    apart (Sec. 2.3: group indices repeat every period)."""
    first: Dict[int, int] = {}
    for p, g in enumerate(patch_group):
        g = int(g)
        if g in first:
            if ((p - first[g]) * w) % period:
                return False
        else:
            first[g] = p
    return True


def roi_pixels(roi: np.ndarray, coils: np.ndarray) -> np.ndarray:
    """Raster (z, y, x) list of ROI pixels that some coil sees (Eq. 7's
    r in ROI; a pixel with sum_n |c_n|^2 = 0 has no encoding vector)."""
    cov = np.sum(np.abs(coils) ** 2, axis=0) > 0
    return np.flatnonzero((roi.astype(bool) & cov).ravel()).astype(np.int64)


def readout_matrix_bytes(ntx_c: int, nx: int, ny: int, nz: int,
                         bytes_per_entry: int = 8) -> int:
    """Size of the explicitly stored compressed readout encoding matrix, one
    N'_tx x N_x block per phase-encode column (SI Table S2)."""
    return ntx_c * nx * ny * nz * bytes_per_entry


# ============================================================ encoding ==

def centred(n: int) -> np.ndarray:
    return np.arange(n) - n // 2


def wave_coeffs(ntx: int, cycles: float, kappa_y: float, kappa_z: float):
    """a_y(t), a_z(t): wave k-space excursion in phase-encode lines (Eq. 3 for
    sinusoidal G_y and cosine G_z)."""
    t = np.arange(ntx, dtype=np.float64)
    th = 2 * PI * cycles * t / ntx
    return kappa_y * (1 - np.cos(th)) / 2, kappa_z * np.sin(th) / 2


def wave_phase(geom) -> np.ndarray:
    """phi(t, z, y) in radians, shape [ntx][nz][ny] (Eq. 3)."""
    ay, az = wave_coeffs(geom.ntx, geom.cycles, geom.kappa_y, geom.kappa_z)
    yc = centred(geom.ny) / geom.ny
    zc = centred(geom.nz) / geom.nz
    return 2 * PI * (ay[:, None, None] * yc[None, None, :]
                     + az[:, None, None] * zc[None, :, None])


def dense_E(geom, coils: np.ndarray) -> np.ndarray:
    """Brute-force encoding matrix (Eq. 1 discretised, Eq. 4): rows (line,
    coil, t), columns raster (z, y, x).  Tiny grids only."""
    nx, ny, nz, nc, ntx = geom.nx, geom.ny, geom.nz, geom.nc, geom.ntx
    L = nx * ny * nz
    zc, yc, xc = np.meshgrid(centred(nz), centred(ny), centred(nx), indexing="ij")
    zc, yc, xc = zc.ravel(), yc.ravel(), xc.ravel()
    z, y = zc + nz // 2, yc + ny // 2
    phi = wave_phase(geom)  # [t][z][y]
    tc = centred(ntx)
    E = np.zeros((geom.n_lines * nc * ntx, L), np.complex128)
    norm = 1.0 / math.sqrt(ntx * ny * nz)
    cmap = coils.reshape(nc, L)
    row = 0
    for ky, kz in zip(geom.line_ky, geom.line_kz):
        kyc, kzc = ky - ny // 2, kz - nz // 2
        for n in range(nc):
            for t in range(ntx):
                ph = (2 * PI * tc[t] * xc / ntx + 2 * PI * kyc * yc / ny
                      + 2 * PI * kzc * zc / nz + phi[t, z, y])
                E[row] = cmap[n] * np.exp(-1j * ph) * norm
                row += 1
    return E


# ---- factorised (matrix-free) encoding: coil multiply -> padded readout DFT
# ---- -> wave PSF -> phase-encode DFT -> line gather (Eq. 1-4 evaluated with
# ---- FFTs; the dense form above pins it).

def _fftc(a, axis):
    return np.fft.fftshift(np.fft.fft(np.fft.ifftshift(a, axes=axis), axis=axis,
                                      norm="ortho"), axes=axis)


def _ifftc(a, axis):
    return np.fft.fftshift(np.fft.ifft(np.fft.ifftshift(a, axes=axis), axis=axis,
                                       norm="ortho"), axes=axis)


def _pad_x(u, ntx):
    nx = u.shape[-1]
    out = np.zeros(u.shape[:-1] + (ntx,), np.complex128)
    s = ntx // 2 - nx // 2
    out[..., s:s + nx] = u
    return out


def _crop_x(u, nx):
    ntx = u.shape[-1]
    s = ntx // 2 - nx // 2
    return u[..., s:s + nx]


def hybrid_forward(geom, coils, rho) -> np.ndarray:
    """Per coil: readout-encoded, wave-modulated hybrid data
    V[n][z][y][t] = e^{-i phi(t,y,z)} * DFT_x{pad(c_n rho)}(t)."""
    u = coils * rho[None]
    U = _fftc(_pad_x(u, geom.ntx), axis=-1)
    psf = np.exp(-1j * wave_phase(geom))  # [t][z][y]
    return U * np.transpose(psf, (1, 2, 0))[None]


def hybrid_adjoint(geom, coils, V) -> np.ndarray:
    psf = np.exp(1j * wave_phase(geom))
    U = V * np.transpose(psf, (1, 2, 0))[None]
    u = _crop_x(_ifftc(U, axis=-1), geom.nx)
    return np.sum(np.conj(coils) * u, axis=0)


def pe_forward(geom, V) -> np.ndarray:
    """Phase-encode DFT over (z, y) and line gather -> [n_lines][...][t]."""
    K = _fftc(_fftc(V, axis=-2), axis=-3)  # [...][kz][ky][t]
    return np.moveaxis(K[..., geom.line_kz, geom.line_ky, :], -2, 0)


def pe_adjoint(geom, S, lead_shape) -> np.ndarray:
    """Scatter lines into a zero-filled (kz, ky) grid and invert the DFT."""
    K = np.zeros(lead_shape + (geom.nz, geom.ny, S.shape[-1]), np.complex128)
    K[..., geom.line_kz, geom.line_ky, :] = np.moveaxis(S, 0, -2)
    return _ifftc(_ifftc(K, axis=-3), axis=-2)


def E_apply(geom, coils, rho) -> np.ndarray:
    """Uncompressed forward model S = E rho (Eq. 4), S[line][coil][t]."""
    return pe_forward(geom, hybrid_forward(geom, coils, rho))


def EH_apply(geom, coils, S) -> np.ndarray:
    """Exact adjoint of E_apply."""
    V = pe_adjoint(geom, S, (geom.nc,))
    return hybrid_adjoint(geom, coils, V)


# ============================================================ compression ==

def encoding_vectors(geom, coils, roi_idx, g_patch: int, T=None) -> np.ndarray:
    """Composite encoding vectors of one patch (Eq. 6): column r of the
    returned N_s x |ROI| matrix is E_g[r], entry (n, tau) =
    c~_n(r) exp(-i [2 pi t_c x_c / N_tx + phi(t, y, z)]), t = p w + tau,
    c~ = T c (noise-decorrelated coil maps).  The phase-encode factor is a
    unit scalar per pixel and cancels in Eq. 9."""
    nx, ny, nz, nc, w = geom.nx, geom.ny, geom.nz, geom.nc, geom.w
    L = nx * ny * nz
    c = coils.reshape(nc, L)
    if T is not None:
        c = T @ c
    c = c[:, roi_idx]
    z = roi_idx // (nx * ny)
    y = (roi_idx // nx) % ny
    x = roi_idx % nx
    xc = x - nx // 2
    phi = wave_phase(geom)
    Eg = np.empty((nc * w, len(roi_idx)), np.complex128)
    for tau in range(w):
        t = g_patch * w + tau
        ph = 2 * PI * (t - geom.ntx // 2) * xc / geom.ntx + phi[t, z, y]
        e = np.exp(-1j * ph)
        for n in range(nc):
            Eg[n * w + tau] = c[n] * e
    return Eg


def gram(geom, coils, roi_idx, g: int, T=None, patch: Optional[int] = None):
    """P_g = (E_g N) E_g^H with N = diag(1 / sum_{N_s} |E_g|^2)
    (Eq. 7, 9, 10, 11), built from the group's first patch unless `patch`
    names another occurrence."""
    if patch is None:
        patch = int(reference_patch(geom.patch_group, geom.n_groups)[g])
    Eg = encoding_vectors(geom, coils, roi_idx, patch, T)
    Nd = 1.0 / np.sum(np.abs(Eg) ** 2, axis=0)
    return (Eg * Nd[None, :]) @ Eg.conj().T


def compression_matrix(P: np.ndarray, keep: int, nc: int, w: int, T=None):
    """Eq. 8 and 12: P_g = U F U^H (eigenvalues descending, ties by index);
    A_g = C_g U^H (T (x) I_w), C_g keeping the first `keep` rows.
    Returns (A_g [keep][N_s], eigenvalues descending)."""
    ev, U = np.linalg.eigh(P)
    order = np.argsort(-ev, kind="stable")
    ev, U = ev[order], U[:, order]
    A = U[:, :keep].conj().T
    if T is not None:
        A = A @ np.kron(T, np.eye(w))
    return A, ev


def keep_from_energy(eigvals, threshold: float, trace=None) -> np.ndarray:
    """Kept dimension per group from the eigenvalue spectrum of P_g (Eq. 8;
    Sec. 2.4: the spectrum quantifies compressibility and indicates N_s').
    Reading: N_s'_g is the smallest k >= 1 whose leading eigenvalues hold
    at least `threshold` of the total, sum_{i<k} max(lambda_i, 0) >=
    threshold * trace_g.  `eigvals` [G][m] holds the leading m eigenvalues
    of each group, descending; trace_g defaults to their sum (all N_s of
    them given) and otherwise is trace(P_g), which is |ROI| for every group
    (each normalised pixel term of Eq. 11 has trace 1).  A group whose m
    leading values do not reach the threshold gets -1."""
    ev = np.asarray(eigvals, dtype=np.float64)
    G = ev.shape[0]
    if trace is None:  # summed in index order, as the running sum below
        tr = []
        for g in range(G):
            t = 0.0
            for k in range(ev.shape[1]):
                t += max(float(ev[g, k]), 0.0)
            tr.append(t)
    else:
        tr = list(np.broadcast_to(np.asarray(trace, dtype=np.float64), (G,)))
    keep = np.full(G, -1, np.int64)
    for g in range(G):
        acc = 0.0
        for k in range(ev.shape[1]):
            acc += max(float(ev[g, k]), 0.0)
            if acc >= threshold * tr[g]:
                keep[g] = k + 1
                break
    return keep


def build_groups(geom, coils, roi, T=None):
    """All groups: (A list, eigenvalue list, P list)."""
    roi_idx = roi_pixels(roi, coils)
    As, evs, Ps = [], [], []
    for g in range(geom.n_groups):
        P = gram(geom, coils, roi_idx, g, T)
        A, ev = compression_matrix(P, int(geom.keep[g]), geom.nc, geom.w, T)
        As.append(A)
        evs.append(ev)
        Ps.append(P)
    return As, evs, Ps


def compress(geom, As, S) -> np.ndarray:
    """S'_{l,p} = A_{g(p)} s_{l,p} (Eq. 13); s_{l,p}[n w + tau] =
    S[l][n][p w + tau]."""
    w, nc = geom.w, geom.nc
    off = patch_offsets(geom.patch_group, geom.keep)
    out = np.zeros((S.shape[0], ntx_compressed(geom.patch_group, geom.keep)),
                   np.complex128)
    for p, g in enumerate(geom.patch_group):
        s = S[:, :, p * w:(p + 1) * w].reshape(S.shape[0], nc * w)
        k = int(geom.keep[g])
        out[:, off[p]:off[p] + k] = s @ As[g].T
    return out


def decompress_adjoint(geom, As, Sc) -> np.ndarray:
    """A^H applied patch by patch: the adjoint of `compress`."""
    w, nc = geom.w, geom.nc
    off = patch_offsets(geom.patch_group, geom.keep)
    out = np.zeros((Sc.shape[0], nc, geom.ntx), np.complex128)
    for p, g in enumerate(geom.patch_group):
        k = int(geom.keep[g])
        s = Sc[:, off[p]:off[p] + k] @ np.conj(As[g])
        out[:, :, p * w:(p + 1) * w] = s.reshape(Sc.shape[0], nc, w)
    return out


def Ec_apply(geom, coils, As, rho) -> np.ndarray:
    """Compressed forward model S'_est = E' rho (Eq. 14-15), as A o E."""
    return compress(geom, As, E_apply(geom, coils, rho))


def EcH_apply(geom, coils, As, Sc) -> np.ndarray:
    return EH_apply(geom, coils, decompress_adjoint(geom, As, Sc))


def readout_Ec_row(geom, coils, As, y: int, z: int = 0) -> np.ndarray:
    """Compressed readout encoding matrix of phase-encode row (y, z)
    (Eq. 14): [N'_tx][N_x], entry (off_p + k, x) = sum_{n, tau}
    A_{g(p)}[k][n w + tau] c_n(z, y, x) exp(-i [2 pi t_c x_c / N_tx +
    phi(t, y, z)]) / sqrt(N_tx), t = p w + tau: the per-column matrix the
    paper stores (SI Table S2)."""
    nx, nc, ntx, w = geom.nx, geom.nc, geom.ntx, geom.w
    xc = centred(nx)
    phi = wave_phase(geom)  # [t][z][y]
    Er = np.zeros((nc, ntx, nx), np.complex128)
    for n in range(nc):
        for t in range(ntx):
            ph = 2 * PI * (t - ntx // 2) * xc / ntx + phi[t, z, y]
            Er[n, t] = coils[n, z, y] * np.exp(-1j * ph) / math.sqrt(ntx)
    off = patch_offsets(geom.patch_group, geom.keep)
    G = np.zeros((ntx_compressed(geom.patch_group, geom.keep), nx), np.complex128)
    for p, g in enumerate(geom.patch_group):
        blk = Er[:, p * w:(p + 1) * w, :].reshape(nc * w, nx)  # rows n w + tau
        k = int(geom.keep[g])
        G[off[p]:off[p] + k] = As[g] @ blk
    return G


def aliased_sets(geom):
    """Phase-encode rows (raster z, y) grouped into the aliased sets of the
    mask: the connected components of the nonzero pattern of
    U = F^H M^T M F, F the centred unitary phase-encode DFT (Sec. 3.4:
    regular / CAIPI masks give R-fold sets of discrete pixels).  Returns
    (sets, F restricted to the sampled lines, U)."""
    ny, nz = geom.ny, geom.nz
    yc = np.tile(centred(ny), nz)
    zc = np.repeat(centred(nz), ny)
    kyc = np.asarray(geom.line_ky) - ny // 2
    kzc = np.asarray(geom.line_kz) - nz // 2
    F = np.exp(-2j * PI * (np.outer(kyc, yc) / ny + np.outer(kzc, zc) / nz)) / math.sqrt(ny * nz)
    U = F.conj().T @ F
    nz_pat = np.abs(U) > 1e-9 * np.abs(U).max()
    parent = list(range(ny * nz))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in zip(*np.nonzero(nz_pat)):
        ra, rb = find(int(a)), find(int(b))
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    sets = {}
    for r in range(ny * nz):
        sets.setdefault(find(r), []).append(r)
    return [sets[k] for k in sorted(sets)], F, U


def decoupled_ls(geom, coils, As, Sc) -> np.ndarray:
    """Hybrid-space reconstruction (Sec. 3.4, algorithm #1) of the least
    squares problem of Eq. 16, in the paper's three steps:
      1. inverse DFT of the zero-filled compressed k-space along the phase
         encode: h~(y, z) = sum_lines F*[line, (y, z)] S'(line);
      2. per aliased set Y (`aliased_sets`), the readout subproblem with the
         |Y| N_x pixels of Y as unknowns and h~ on Y as data: its normal
         equations sum_{r''} G_r^H U[r, r''] G_r'' rho_r'' = G_r^H h~(r),
         r, r'' in Y, with G_r the row's compressed readout matrix, solved by
         least squares (minimum norm where singular);
      3. assemble the rows of all sets into the image.
    The sets decouple the normal equations exactly (U vanishes between
    them), so this is the global least-squares solution; regular and CAIPI
    masks give sets of R pixels."""
    nx, ny, nz = geom.nx, geom.ny, geom.nz
    sets, F, U = aliased_sets(geom)
    ht = F.conj().T @ Sc  # step 1: [rows][N'_tx]
    Gs = [readout_Ec_row(geom, coils, As, r % ny, r // ny) for r in range(ny * nz)]
    rho = np.zeros((ny * nz, nx), np.complex128)
    for Y in sets:  # step 2
        m = len(Y)
        N = np.zeros((m * nx, m * nx), np.complex128)
        b = np.zeros(m * nx, np.complex128)
        for a, ra in enumerate(Y):
            b[a * nx:(a + 1) * nx] = Gs[ra].conj().T @ ht[ra]
            for c, rb in enumerate(Y):
                N[a * nx:(a + 1) * nx, c * nx:(c + 1) * nx] = Gs[ra].conj().T @ (U[ra, rb] * Gs[rb])
        sol = np.linalg.lstsq(N, b, rcond=None)[0]
        for a, ra in enumerate(Y):  # step 3
            rho[ra] = sol[a * nx:(a + 1) * nx]
    return rho.reshape(nz, ny, nx)


def decoupled_cg(geom, coils, As, Sc, iters: int) -> np.ndarray:
    """Algorithm #1 (Sec. 3.4) with an iterative solver per readout
    subproblem, the form the paper runs (LSQR per aliased set): steps 1 and
    3 as in `decoupled_ls`; in step 2 every aliased set Y solves its own
    normal equations N_Y rho_Y = b_Y by CG with its own scalars, exactly
    `iters` iterations (stopping early only when ||r_Y||^2 == 0; CG on the
    normal equations has LSQR's iterates in exact arithmetic)."""
    nx, ny, nz = geom.nx, geom.ny, geom.nz
    sets, F, U = aliased_sets(geom)
    ht = F.conj().T @ Sc  # step 1
    Gs = [readout_Ec_row(geom, coils, As, r % ny, r // ny) for r in range(ny * nz)]
    rho = np.zeros((ny * nz, nx), np.complex128)
    for Y in sets:  # step 2: the set's own normal equations and CG
        m = len(Y)
        N = np.zeros((m * nx, m * nx), np.complex128)
        b = np.zeros(m * nx, np.complex128)
        for a, ra in enumerate(Y):
            b[a * nx:(a + 1) * nx] = Gs[ra].conj().T @ ht[ra]
            for c, rb in enumerate(Y):
                N[a * nx:(a + 1) * nx, c * nx:(c + 1) * nx] = Gs[ra].conj().T @ (U[ra, rb] * Gs[rb])
        sol, _ = cg(lambda v: N @ v, b, iters)
        for a, ra in enumerate(Y):  # step 3
            rho[ra] = sol[a * nx:(a + 1) * nx]
    return rho.reshape(nz, ny, nx)


def dense_Ec(geom, coils, As) -> np.ndarray:
    """E' = A E (Eq. 14) as a dense matrix (tiny grids only)."""
    E = dense_E(geom, coils)
    nl, nc, ntx, w = geom.n_lines, geom.nc, geom.ntx, geom.w
    E = E.reshape(nl, nc, ntx, -1)
    off = patch_offsets(geom.patch_group, geom.keep)
    ntxc = ntx_compressed(geom.patch_group, geom.keep)
    out = np.zeros((nl, ntxc, E.shape[-1]), np.complex128)
    for p, g in enumerate(geom.patch_group):
        blk = E[:, :, p * w:(p + 1) * w, :].reshape(nl, nc * w, -1)
        out[:, off[p]:off[p] + int(geom.keep[g]), :] = np.einsum(
            "ki,lir->lkr", As[g], blk)
    return out.reshape(nl * ntxc, -1)


# ============================================================ reconstruction ==

def cg(normal: Callable, b: np.ndarray, iters: int, x0=None, fwd=None,
       adj=None):
    """CG on the normal equations E'^H E' x = E'^H S' (Sec. 3.4, Eq. 16),
    exactly `iters` iterations, stopping early only when ||r||^2 == 0:
      alpha = ||r||^2 / ||E' p||^2, x += alpha p, r -= alpha E'^H E' p,
      beta = ||r_new||^2 / ||r||^2, p = r + beta p.
    With `fwd` and `adj` the product is formed as adj(fwd(p)) and the
    denominator as ||fwd(p)||^2; otherwise as normal(p) and <p, normal(p)>.
    Returns (x, [||r||^2 at the start of each iteration and at the end])."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - normal(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    hist = [rr]
    for _ in range(iters):
        if rr == 0.0:
            break
        if fwd is not None and adj is not None:
            q = fwd(p)
            Ap = adj(q)
            den = np.vdot(q, q).real
        else:
            Ap = normal(p)
            den = np.vdot(p, Ap).real
        alpha = rr / den
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        hist.append(rr)
    return x, hist


def haar_fwd(img: np.ndarray, levels: int) -> np.ndarray:
    """Orthonormal 2D Haar transform, `levels` levels, Mallat layout
    (approximation top-left).  img is [ny][nx] (or [..., ny, nx])."""
    out = img.astype(np.complex128).copy()
    h, w = out.shape[-2:]
    s = 1.0 / math.sqrt(2.0)
    for _ in range(levels):
        blk = out[..., :h, :w].copy()
        lo = (blk[..., :, 0::2] + blk[..., :, 1::2]) * s
        hi = (blk[..., :, 0::2] - blk[..., :, 1::2]) * s
        blk = np.concatenate([lo, hi], axis=-1)
        lo = (blk[..., 0::2, :] + blk[..., 1::2, :]) * s
        hi = (blk[..., 0::2, :] - blk[..., 1::2, :]) * s
        out[..., :h, :w] = np.concatenate([lo, hi], axis=-2)
        h //= 2
        w //= 2
    return out


def haar_inv(coef: np.ndarray, levels: int) -> np.ndarray:
    out = coef.astype(np.complex128).copy()
    H, W = out.shape[-2:]
    s = 1.0 / math.sqrt(2.0)
    for lev in reversed(range(levels)):
        h, w = H >> lev, W >> lev
        blk = out[..., :h, :w].copy()
        lo, hi = blk[..., : h // 2, :], blk[..., h // 2:, :]
        rows = np.empty_like(blk)
        rows[..., 0::2, :] = (lo + hi) * s
        rows[..., 1::2, :] = (lo - hi) * s
        lo, hi = rows[..., :, : w // 2], rows[..., :, w // 2:]
        cols = np.empty_like(rows)
        cols[..., :, 0::2] = (lo + hi) * s
        cols[..., :, 1::2] = (lo - hi) * s
        out[..., :h, :w] = cols
    return out


def soft(z: np.ndarray, tau: float) -> np.ndarray:
    """Complex soft threshold z * max(0, 1 - tau/|z|), soft(0) = 0."""
    mag = np.abs(z)
    scale = np.where(mag > tau, 1.0 - tau / np.where(mag > 0, mag, 1.0), 0.0)
    return z * scale


def detail_mask(ny: int, nx: int, levels: int) -> np.ndarray:
    """True on detail (thresholded) coefficients, False on the coarsest
    approximation block."""
    m = np.ones((ny, nx), bool)
    m[: ny >> levels, : nx >> levels] = False
    return m


def wavelet_prox(z2d: np.ndarray, tau: float, levels: int) -> np.ndarray:
    """W^H soft_tau(W z) with the threshold on detail bands only."""
    c = haar_fwd(z2d, levels)
    m = detail_mask(z2d.shape[-2], z2d.shape[-1], levels)
    c = np.where(m, soft(c, tau), c)
    return haar_inv(c, levels)


def power_lipschitz(normal: Callable, v0: np.ndarray, iters: int) -> float:
    """Largest eigenvalue of E'^H E' by power iteration: v <- N v / ||N v||;
    returns the final ||N v|| with ||v|| = 1."""
    v = v0 / np.linalg.norm(v0)
    L = 0.0
    for _ in range(iters):
        u = normal(v)
        L = float(np.linalg.norm(u))
        v = u / L
    return L


def tv_diff(u):
    """Forward differences of a 2D image along x and y, zero across the last
    column / row (Neumann boundary)."""
    dx = np.zeros_like(u)
    dy = np.zeros_like(u)
    dx[:, :-1] = u[:, 1:] - u[:, :-1]
    dy[:-1, :] = u[1:, :] - u[:-1, :]
    return dx, dy


def tv_diff_adj(px, py):
    """Adjoint of `tv_diff`: (D_x^H p_x + D_y^H p_y)."""
    out = np.zeros_like(px)
    out[:, :-1] -= px[:, :-1]
    out[:, 1:] += px[:, :-1]
    out[:-1, :] -= py[:-1, :]
    out[1:, :] += py[:-1, :]
    return out


def tv_smooth(u: np.ndarray, eps: float) -> float:
    """Smoothed isotropic total variation of a 2D image (Eq. 17's TV term,
    by a smooth approximation as Sec. 3.4 states):
    sum_{y,x} sqrt(|D_x u|^2 + |D_y u|^2 + eps^2)."""
    dx, dy = tv_diff(u)
    return float(np.sum(np.sqrt(np.abs(dx) ** 2 + np.abs(dy) ** 2 + eps * eps)))


def tv_smooth_grad(u: np.ndarray, eps: float) -> np.ndarray:
    """Gradient of `tv_smooth` with respect to the real and imaginary parts,
    as one complex image: D^H (D u / sqrt(|D u|^2 + eps^2)).  It is
    Lipschitz with constant ||D||^2 / eps <= 8 / eps."""
    dx, dy = tv_diff(u)
    wgt = np.sqrt(np.abs(dx) ** 2 + np.abs(dy) ** 2 + eps * eps)
    return tv_diff_adj(dx / wgt, dy / wgt)


def fista(normal: Callable, b: np.ndarray, L: float, lam: float, levels: int,
          iters: int, x0=None, lam_tv: float = 0.0, eps_tv: float = 1e-3) -> np.ndarray:
    """FISTA (Beck-Teboulle) for 1/2 ||E' x - S'||^2 + lam ||W x||_1 on the
    detail bands + lam_tv TV_eps(x) (Eq. 17, TV by its smooth approximation,
    which joins the gradient step):
      x_k = W^H soft_{lam/L}(W (y_k - (E'^H E' y_k - E'^H S'
                                      + lam_tv grad TV_eps(y_k)) / L)),
      t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
      y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1}).
    L must bound the Lipschitz constant of the whole gradient (that of
    E'^H E' plus 8 lam_tv / eps_tv).  Images are [nz][ny][nx]; the 2D
    transforms run per z-slice."""
    x_prev = np.zeros_like(b) if x0 is None else x0.copy()
    y = x_prev.copy()
    t = 1.0
    for _ in range(iters):
        grad = normal(y) - b
        if lam_tv != 0.0:
            grad = grad + lam_tv * np.stack([tv_smooth_grad(y[k], eps_tv) for k in range(y.shape[0])])
        z = y - grad / L
        x = np.stack([wavelet_prox(z[k], lam / L, levels) for k in range(z.shape[0])])
        t_new = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        y = x + ((t - 1.0) / t_new) * (x - x_prev)
        x_prev, t = x, t_new
    return x_prev


def nrmse(x: np.ndarray, ref: np.ndarray) -> float:
    """NRMSE normalised by the reference range, max - min (Sec. 3.4), on the
    complex values over the full grid."""
    d = np.linalg.norm((x - ref).ravel()) / math.sqrt(ref.size)
    a = np.abs(ref)
    return float(d / (a.max() - a.min()))


def nrmse_mag(x: np.ndarray, ref: np.ndarray) -> float:
    a = np.abs(ref)
    d = np.linalg.norm((np.abs(x) - a).ravel()) / math.sqrt(ref.size)
    return float(d / (a.max() - a.min()))


# ============================================================ pipeline ==

# ============================================== nonlinear B0 modulation ==
# Local B0 coils (Sec. 2.1-2.2, Eq. 2-3): the modulation phase depends on the
# readout position as well, phi(t, r) = sum_lambda a_lambda(t) B_lambda(r),
# so the readout is no longer a DFT and the compressed readout encoding of
# each phase-encode row is a stored matrix (Eq. 14).  The phase-encode DFT
# still factors out because phi does not depend on the phase-encode step.

def local_b0_phase(fields: np.ndarray, amps: np.ndarray) -> np.ndarray:
    """phi[t][z][y][x] = sum_lambda amps[lambda][t] fields[lambda][z][y][x]
    (radians): the time-varying fields of the local B0 coils (Eq. 2-3)."""
    return np.einsum("lt,lzyx->tzyx", np.asarray(amps, np.float64), np.asarray(fields, np.float64))


def dense_E_phase(geom, coils: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Brute-force encoding matrix (Eq. 1, 4) for a general modulation phase
    phi[t][z][y][x]: rows (line, coil, t), columns raster (z, y, x)."""
    nx, ny, nz, nc, ntx = geom.nx, geom.ny, geom.nz, geom.nc, geom.ntx
    L = nx * ny * nz
    zc, yc, xc = np.meshgrid(centred(nz), centred(ny), centred(nx), indexing="ij")
    zc, yc, xc = zc.ravel(), yc.ravel(), xc.ravel()
    ph_r = phi.reshape(ntx, L)
    tc = centred(ntx)
    E = np.zeros((geom.n_lines * nc * ntx, L), np.complex128)
    norm = 1.0 / math.sqrt(ntx * ny * nz)
    cmap = coils.reshape(nc, L)
    row = 0
    for ky, kz in zip(geom.line_ky, geom.line_kz):
        kyc, kzc = ky - ny // 2, kz - nz // 2
        for n in range(nc):
            for t in range(ntx):
                ph = (2 * PI * tc[t] * xc / ntx + 2 * PI * kyc * yc / ny
                      + 2 * PI * kzc * zc / nz + ph_r[t])
                E[row] = cmap[n] * np.exp(-1j * ph) * norm
                row += 1
    return E


def readout_row_phase(geom, coils, As, phi: np.ndarray, y: int, z: int = 0) -> np.ndarray:
    """Compressed readout encoding matrix E'_g of phase-encode row (y, z) for
    a general phase (Eq. 14): [N'_tx][N_x], entry (off_p + k, x) =
    sum_{n,tau} A_{g(p)}[k][n w + tau] c_n(z,y,x)
    exp(-i [2 pi t_c x_c / N_tx + phi(t,z,y,x)]) / sqrt(N_tx), t = p w + tau."""
    nx, nc, ntx, w = geom.nx, geom.nc, geom.ntx, geom.w
    xc = centred(nx)
    Er = np.zeros((nc, ntx, nx), np.complex128)
    for n in range(nc):
        for t in range(ntx):
            ph = 2 * PI * (t - ntx // 2) * xc / ntx + phi[t, z, y, :]
            Er[n, t] = coils[n, z, y] * np.exp(-1j * ph) / math.sqrt(ntx)
    off = patch_offsets(geom.patch_group, geom.keep)
    G = np.zeros((ntx_compressed(geom.patch_group, geom.keep), nx), np.complex128)
    for p, g in enumerate(geom.patch_group):
        k = int(geom.keep[g])
        G[off[p]:off[p] + k] = As[g] @ Er[:, p * w:(p + 1) * w, :].reshape(nc * w, nx)
    return G


def Ec_apply_phase(geom, coils, As, phi: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """E' rho for a general phase: every row's stored readout matrix, then
    the centred unitary phase-encode DFT and the line gather (Eq. 14-15)."""
    nx, ny, nz = geom.nx, geom.ny, geom.nz
    H = np.stack([readout_row_phase(geom, coils, As, phi, r % ny, r // ny) @ rho[r // ny, r % ny]
                  for r in range(ny * nz)])  # [rows][N'_tx]
    yc = np.tile(centred(ny), nz)
    zc = np.repeat(centred(nz), ny)
    kyc = np.asarray(geom.line_ky) - ny // 2
    kzc = np.asarray(geom.line_kz) - nz // 2
    F = np.exp(-2j * PI * (np.outer(kyc, yc) / ny + np.outer(kzc, zc) / nz)) / math.sqrt(ny * nz)
    return F @ H


def dense_Ec_phase(geom, coils, As, phi: np.ndarray) -> np.ndarray:
    """E' = A E (Eq. 14) for a general phase as a dense matrix (tiny grids
    only): rows (line, off_p + k), columns raster (z, y, x)."""
    E = dense_E_phase(geom, coils, phi)
    nl, nc, ntx, w = geom.n_lines, geom.nc, geom.ntx, geom.w
    E = E.reshape(nl, nc, ntx, -1)
    off = patch_offsets(geom.patch_group, geom.keep)
    out = np.zeros((nl, ntx_compressed(geom.patch_group, geom.keep), E.shape[-1]), np.complex128)
    for p, g in enumerate(geom.patch_group):
        blk = E[:, :, p * w:(p + 1) * w, :].reshape(nl, nc * w, -1)
        out[:, off[p]:off[p] + int(geom.keep[g]), :] = np.einsum("ki,lir->lkr", As[g], blk)
    return out.reshape(nl * ntx_compressed(geom.patch_group, geom.keep), -1)


def gram_phase(geom, coils, roi_idx, g: int, phi: np.ndarray, T=None) -> np.ndarray:
    """P_g (Eq. 7-11) for a general phase: encoding vectors of the group's
    first patch, entry (n, tau) = c~_n(r) exp(-i [2 pi t_c x_c / N_tx +
    phi(t, r)]), normalised per pixel."""
    nx, ny, nc, w = geom.nx, geom.ny, geom.nc, geom.w
    L = nx * ny * geom.nz
    c = coils.reshape(nc, L)
    if T is not None:
        c = T @ c
    c = c[:, roi_idx]
    xc = roi_idx % nx - nx // 2
    ph_r = phi.reshape(geom.ntx, L)[:, roi_idx]
    patch = int(reference_patch(geom.patch_group, geom.n_groups)[g])
    Eg = np.empty((nc * w, len(roi_idx)), np.complex128)
    for tau in range(w):
        t = patch * w + tau
        e = np.exp(-1j * (2 * PI * (t - geom.ntx // 2) * xc / geom.ntx + ph_r[t]))
        for n in range(nc):
            Eg[n * w + tau] = c[n] * e
    Nd = 1.0 / np.sum(np.abs(Eg) ** 2, axis=0)
    return (Eg * Nd[None, :]) @ Eg.conj().T


class Problem:
    """Convenience bundle: operators bound to one geometry and coil set."""

    def __init__(self, geom, coils, As=None):
        self.g, self.c, self.As = geom, coils, As

    def E(self, x):
        return E_apply(self.g, self.c, x)

    def EH(self, s):
        return EH_apply(self.g, self.c, s)

    def Ec(self, x):
        return Ec_apply(self.g, self.c, self.As, x)

    def EcH(self, s):
        return EcH_apply(self.g, self.c, self.As, s)

    def normal_c(self, x):
        return self.EcH(self.Ec(x))


def simulate(geom, coils, rho, noise) -> np.ndarray:
    """Raw k-space S = E rho + n (Eq. 4 with additive receiver noise)."""
    return E_apply(geom, coils, rho) + noise


def reconstruct(geom, coils, As, Sc, alg: str, iters: int, lam: float = 0.0,
                levels: int = 4, L: Optional[float] = None,
                v0: Optional[np.ndarray] = None, power_iters: int = 50):
    """End-to-end compressed reconstruction on given compressed data."""
    pb = Problem(geom, coils, As)
    b = pb.EcH(Sc)
    if alg == "cg":
        x, _ = cg(pb.normal_c, b, iters, fwd=pb.Ec, adj=pb.EcH)
        return x, None
    if L is None:
        L = power_lipschitz(pb.normal_c, v0, power_iters)
    return fista(pb.normal_c, b, L, lam, levels, iters), L
