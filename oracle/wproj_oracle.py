"""FP64 CPU oracle for the sparse w-projection hot path (Wolz et al. 2013).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package entry
file and the CPU-baseline leg of the benchmark may import this module.  The
product (the CUDA library and its Python binding) never calls it, and it shares
no code, table or constant generator with the CUDA path.

Everything here is plain, slow and written to be checked against the paper by
eye: complex128 / float64 NumPy, with numpy.fft and scipy.sparse as the only
library primitives.  Each function cites the passage it follows.

Model (the paper's operator, Eq. 8, with continuous (u, v) and a
Kaiser-Bessel gridding kernel):

    Phi = G . F . Z . A

  A  diagonal correction 1/(a(l) a(m)), a = Fourier transform of the KB kernel
  Z  centred zero-padding of the N x N image onto the 2N x 2N grid
  F  unitary 2-D DFT (1/G normalisation, e^{-2 pi i ...} sign of Eq. 1)
  G  sparse rows: for visibility k, the w-modulation kernel C-hat of Eq. 8
     (Section 3.1: FFT of the real-space chirp, Eq. 4), convolved with the KB
     taps at the visibility's sub-grid offset, then sparsified per row by the
     adaptive energy threshold of Section 3.2.

Readings of the paper taken here (the paper is silent or inconsistent):
  * 1/n of Eq. 1 is absorbed into the image (x := I/n), as Eq. 6 omits it.
  * Eq. 5 prints exp(-pi i w r^2) while the first-order expansion of Eq. 4
    gives exp(+pi i w r^2); the '+' sign (consistent with Eq. 4) is used.
  * "Energy" of a row is the sum of squared moduli of the KB-convolved row;
    entries are ordered by modulus, ties broken by the lower column index;
    the kept set is the shortest prefix whose exactly rounded sum reaches
    e * E.  No renormalisation after truncation.
  * The chirp is sampled on an S x S box spanning [-L, L)^2 (S = G is exact);
    outside the field of view it is either evaluated as is ('full') or with
    the coordinates clamped to the field of view ('clamp').
  * Direction-dependent effects (Section 3.2 claims the per-row threshold
    applies to all of them): a screen A(l, m) per visibility multiplies the
    chirp in image space before the FFT, sampled at the same G x G points.
  * KB: W = 4, oversampling 2, beta from Beatty, Nishimura & Pauly (2005);
    taps at j0-W/2+1 .. j0+W/2 (half-open at a cell boundary).

Indexing conventions: grid arrays are G x G in natural FFT order (frequency q
stored at index q mod G).  The image pixel p in [0, N) sits at offset
p - N/2, i.e. at padded index (p - N/2) mod G.  Column of grid cell (qu, qv)
is (qu mod G) * G + (qv mod G).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse
import scipy.special

# ----------------------------------------------------------------------------
# Kaiser-Bessel gridding kernel and its Fourier transform (the gridding used here;
# Jackson et al. 1991, Beatty et al. 2005).  Not in the paper itself, which
# keeps visibilities on the grid (Section 2.2).
# ----------------------------------------------------------------------------


def kb_beta(W: int = 4, sigma: float = 2.0) -> float:
    """beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8) (Beatty et al. 2005)."""
    return math.pi * math.sqrt((W / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)


def kb(t, W: int, beta: float):
    """kb(t) = I0(beta sqrt(1 - (2t/W)^2)) for |t| <= W/2, else 0."""
    t = np.asarray(t, dtype=np.float64)
    arg = 1.0 - (2.0 * t / W) ** 2
    out = np.where(arg >= 0.0, scipy.special.i0(beta * np.sqrt(np.maximum(arg, 0.0))), 0.0)
    return out


def kb_ft(nu, W: int, beta: float):
    """Continuous Fourier transform of kb at frequency nu:
    W sinh(sqrt(beta^2 - (pi W nu)^2)) / sqrt(...), with the sin branch when
    the radicand is negative (Jackson et al. 1991)."""
    nu = np.asarray(nu, dtype=np.float64)
    z2 = beta * beta - (math.pi * W * nu) ** 2
    out = np.empty_like(nu)
    pos = z2 > 0
    neg = z2 < 0
    zer = ~(pos | neg)
    zp = np.sqrt(z2[pos])
    out[pos] = W * np.sinh(zp) / zp
    zn = np.sqrt(-z2[neg])
    out[neg] = W * np.sin(zn) / zn
    out[zer] = W
    return out


def taps(W: int):
    """Tap offsets t relative to j0 = floor(g): {-W/2+1, ..., W/2}; a single
    tap {0} for delta-gridding (W = 1)."""
    if W == 1:
        return np.array([0])
    return np.arange(-W // 2 + 1, W // 2 + 1)


def tap_weights(delta: float, W: int, beta: float):
    """kb(delta - t) for the taps t (delta = g - floor(g) in [0, 1))."""
    if W == 1:
        return np.array([1.0])
    return kb(delta - taps(W), W, beta)


def correction(N: int, W: int, beta: float):
    """a(l_p) for the image pixels p in [0, N): nu = l_p du = (p - N/2) / (2N).
    For delta-gridding (W = 1), a = 1."""
    if W == 1:
        return np.ones(N)
    nu = (np.arange(N) - N // 2) / (2.0 * N)
    return kb_ft(nu, W, beta)


# ----------------------------------------------------------------------------
# w-modulation chirp (Section 2.1, Eqs. 4 and 5)
# ----------------------------------------------------------------------------


def chirp(l, m, w: float, kind: str = "exact"):
    """C(l, m; w) of Eq. 4: exp(-2 pi i w (n - 1)) = exp(2 pi i w (1 - n)),
    n = sqrt(1 - l^2 - m^2); 1 - n is evaluated as r^2 / (1 + n) to avoid
    cancellation.  kind='linear' is Eq. 5 with the '+' sign reading."""
    r2 = np.asarray(l, dtype=np.float64) ** 2 + np.asarray(m, dtype=np.float64) ** 2
    if kind == "exact":
        if np.any(r2 > 1.0):
            raise ValueError("1 - l^2 - m^2 < 0 on the sampled box")
        one_minus_n = r2 / (1.0 + np.sqrt(1.0 - r2))
        return np.exp(2j * np.pi * w * one_minus_n)
    if kind == "linear":
        return np.exp(1j * np.pi * w * r2)
    raise ValueError(kind)


def box_coords(S: int, L: float, extension: str = "full"):
    """S sample positions per axis spanning [-L, L): l'_P = (P - S/2) 2L/S.
    'clamp' clamps them to the field of view [-L/2, L/2]."""
    lp = (np.arange(S) - S // 2) * (2.0 * L / S)
    if extension == "clamp":
        lp = np.clip(lp, -L / 2.0, L / 2.0)
    elif extension != "full":
        raise ValueError(extension)
    return lp


def centred_dft2(a):
    """Unitary centred 2-D DFT of an S x S array whose index P holds offset
    P - S/2; returns natural order (frequency m at index m mod S):
    A[m] = (1/S) sum_P a[P] exp(-2 pi i m . (P - S/2) / S)."""
    S = a.shape[0]
    return np.fft.fft2(np.fft.ifftshift(a)) / S


def direct_centred_dft2(a):
    """The same transform as `centred_dft2` by explicit summation (for pins)."""
    S = a.shape[0]
    off = np.arange(S) - S // 2
    m = np.arange(S)
    E = np.exp(-2j * np.pi * np.outer(m, off) / S)
    return E @ a @ E.T / S


# ----------------------------------------------------------------------------
# Kernel rows of G (Sections 3.1 and 3.2, Eq. 8)
# ----------------------------------------------------------------------------


class Geometry:
    """N x N image, G = 2N grid, field of view L, KB support W."""

    def __init__(self, N: int, L: float, W: int = 4, sigma: float = 2.0,
                 chirp_kind: str = "exact", extension: str = "full"):
        self.N = N
        self.G = 2 * N
        self.L = L
        self.W = W
        self.beta = kb_beta(W, sigma) if W > 1 else 0.0
        self.dl = L / N
        self.du = 1.0 / (2.0 * L)
        self.chirp_kind = chirp_kind
        self.extension = extension
        self.a = correction(N, W, self.beta)


def kernel_box(geo: Geometry, u: float, v: float, w: float, S: int, screen=None):
    """Unthresholded kernel of one visibility on its S x S box.

    Returns (K, j0u, j0v) with K[su mod S, sv mod S] the weight of grid cell
    (j0u + su, j0v + sv) for the centred box offsets s in [-S/2, S/2)^2, i.e.

      G[k, j0 + s] = (1/S) sum_t T[t] Chat[t - s]     (indices mod S)

    Chat = unitary centred DFT of the chirp sampled on the box (the row of
    C-hat of Eq. 8, Section 3.2: chirp in real space, then a 2-D FFT),
    T[t] = kb(du - tu) kb(dv - tv) the gridding taps at the sub-grid offset.
    At S = G this is the exact circular convolution of C-hat with the taps.

    screen: an optional direction-dependent effect (Section 3.2: the threshold
    makes no assumption on a row's structure, so it applies to any such
    effect): a G x G complex array sampled at the chirp's points, index P
    holding offset P - G/2 (pixel p of the image sits at index p + N/2).  The
    row is then the FFT of (chirp x screen), convolved with the taps.  Needs S = G.
    """
    gu, gv = u / geo.du, v / geo.du
    j0u, j0v = math.floor(gu), math.floor(gv)
    tu = tap_weights(gu - j0u, geo.W, geo.beta)
    tv = tap_weights(gv - j0v, geo.W, geo.beta)
    lp = box_coords(S, geo.L, geo.extension)
    c = chirp(lp[:, None], lp[None, :], w, geo.chirp_kind)
    if screen is not None:
        screen = np.asarray(screen)
        if S != geo.G or screen.shape != (S, S):
            raise ValueError("a screen needs the full box S = G and a G x G array")
        c = c * screen
    Chat = centred_dft2(c)
    # R[s] = Chat[-s]; then Chat[t - s] = R[s - t] = roll(R, t)[s]
    R = np.roll(Chat[::-1, ::-1], 1, axis=(0, 1))
    K = np.zeros((S, S), dtype=np.complex128)
    for a_, ta in enumerate(taps(geo.W)):
        for b_, tb in enumerate(taps(geo.W)):
            K += tu[a_] * tv[b_] * np.roll(R, (int(ta), int(tb)), axis=(0, 1))
    K /= S
    return K, j0u, j0v


def box_columns(geo: Geometry, j0u: int, j0v: int, S: int):
    """Absolute column of each box entry, same layout as K (natural order)."""
    s = np.fft.fftfreq(S, 1.0 / S).astype(np.int64)   # offset held at index s mod S
    qu = (j0u + s) % geo.G
    qv = (j0v + s) % geo.G
    return qu[:, None] * geo.G + qv[None, :]


def energy_closed_form(geo: Geometry, u: float, v: float):
    """Parseval with |c| = 1: E = (sum_t kb(du - t)^2)(sum_t kb(dv - t)^2)."""
    gu, gv = u / geo.du, v / geo.du
    tu = tap_weights(gu - math.floor(gu), geo.W, geo.beta)
    tv = tap_weights(gv - math.floor(gv), geo.W, geo.beta)
    return float(np.sum(tu ** 2) * np.sum(tv ** 2))


# ----------------------------------------------------------------------------
# Adaptive sparsification (Section 3.2)
# ----------------------------------------------------------------------------


def _prefix_reaches(p_sorted, n, target):
    return math.fsum(p_sorted[:n]) >= target


def select_sort(values, cols, e: float):
    """Smallest set of entries whose energy (sum of |.|^2) reaches e * E,
    E the sum over the whole row (Section 3.2).  Entries are taken by
    decreasing modulus, ties by increasing column.  The decision uses an
    exactly rounded sum (math.fsum).  Returns the kept positions (into the
    flattened arrays) in the order taken."""
    p = np.abs(np.asarray(values).ravel()) ** 2
    cols = np.asarray(cols).ravel()
    E = math.fsum(p)
    target = e * E
    order = np.lexsort((cols, -p))
    ps = p[order]
    if not (target > 0.0):
        return order[:0]
    # approximate cut from the running sum, then settle it with fsum
    cs = np.cumsum(ps)
    n = int(np.searchsorted(cs, target, side="left")) + 1
    n = min(max(n, 1), ps.size)
    while n < ps.size and not _prefix_reaches(ps, n, target):
        n += 1
    while n > 1 and _prefix_reaches(ps, n - 1, target):
        n -= 1
    return order[:n]


def select_bisect(values, e: float, iters: int = 200):
    """The paper's route (Section 3.2): threshold tau on |.|, kept set
    {|K| >= tau}, tau found by bisection so that the kept energy reaches e*E
    with tau as large as possible.  Returns a boolean mask."""
    a = np.abs(np.asarray(values).ravel())
    p = a ** 2
    E = math.fsum(p)
    target = e * E

    def kept_energy(tau):
        return math.fsum(p[a >= tau])

    lo, hi = 0.0, float(a.max())     # energy(lo) = E >= target
    if kept_energy(hi) >= target:
        return a >= hi
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if kept_energy(mid) >= target:
            lo = mid
        else:
            hi = mid
    return a >= lo


# ----------------------------------------------------------------------------
# G as a sparse matrix
# ----------------------------------------------------------------------------


def kernel_row(geo: Geometry, u: float, v: float, w: float, S: int, e: float, screen=None):
    """Sparse row k of G: (columns ascending, values) after thresholding."""
    K, j0u, j0v = kernel_box(geo, u, v, w, S, screen)
    cols = box_columns(geo, j0u, j0v, S)
    kept = select_sort(K, cols, e)
    c = cols.ravel()[kept]
    val = K.ravel()[kept]
    o = np.argsort(c)
    return c[o], val[o]


def row_box(geo: Geometry, w: float, S) -> int:
    """Box side of one row: S = None -> G (exact), 'rule' -> S(w) with the
    chirp half-band h = |w| L^2 cells, an int -> that fixed size."""
    if S is None:
        return geo.G
    if S == "rule":
        return box_size_rule(geo, abs(w) * geo.L * geo.L)
    return int(S)


def build_G(geo: Geometry, uvw: np.ndarray, e: float, S=None, screens=None, screen_id=None):
    """CSR G (M x G^2, complex128), one thresholded kernel per visibility.
    screens (n x G x G) with screen_id (M ints) attach a direction-dependent
    screen to every row (kernel_box); then S must be None (the full box)."""
    M = uvw.shape[0]
    rows, cols, vals = [], [], []
    ptr = [0]
    for k in range(M):
        Sk = row_box(geo, uvw[k, 2], S)
        scr = None if screens is None else screens[int(screen_id[k])]
        c, v = kernel_row(geo, uvw[k, 0], uvw[k, 1], uvw[k, 2], Sk, e, scr)
        cols.append(c)
        vals.append(v)
        ptr.append(ptr[-1] + c.size)
    data = np.concatenate(vals) if vals else np.zeros(0, complex)
    ind = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    return scipy.sparse.csr_matrix((data, ind, np.array(ptr)), shape=(M, geo.G * geo.G))


def box_size_rule(geo: Geometry, h: float) -> int:
    """S(w) = min(G, smallest power of two >= 4h + W + 16), h the chirp
    half-bandwidth in uv cells."""
    need = 4.0 * h + geo.W + 16
    S = 1
    while S < need:
        S *= 2
    return min(geo.G, S)


# ----------------------------------------------------------------------------
# Operators (Eq. 6 / Eq. 8 with Z, A and KB gridding)
# ----------------------------------------------------------------------------


def _image_index(geo: Geometry):
    return (np.arange(geo.N) - geo.N // 2) % geo.G


def AZ(geo: Geometry, x):
    """Z A x: divide by a(l) a(m), place the N x N image centred on the G x G
    grid (offset p - N/2 at padded index (p - N/2) mod G), zeros elsewhere."""
    xp = np.zeros((geo.G, geo.G), dtype=np.complex128)
    idx = _image_index(geo)
    xp[np.ix_(idx, idx)] = np.asarray(x) / np.outer(geo.a, geo.a)
    return xp


def AZ_adj(geo: Geometry, xp):
    """(Z A)^H: crop the centred N x N block and divide by a(l) a(m)."""
    idx = _image_index(geo)
    return xp[np.ix_(idx, idx)] / np.outer(geo.a, geo.a)


def F(geo: Geometry, xp):
    """Unitary 2-D DFT on the G x G grid, natural order."""
    return np.fft.fft2(xp) / geo.G


def F_adj(geo: Geometry, X):
    return np.fft.ifft2(X) * geo.G


def phi(geo: Geometry, Gm, x):
    """Phi x = G F Z A x."""
    return Gm @ F(geo, AZ(geo, x)).ravel()


def phi_adj(geo: Geometry, Gm, y):
    """Phi^H y = A Z^H F^H G^H y (complex image); G^H y = conj(G^T conj(y))."""
    Xt = np.conj(Gm.T @ np.conj(np.asarray(y))).reshape(geo.G, geo.G)
    return AZ_adj(geo, F_adj(geo, Xt))


# ----------------------------------------------------------------------------
# Paper mode: the paper's own operator Phi' = C-hat F U of Section 2.2 (Eq. 8)
# for visibilities on the grid: U upsamples the N x N image by zero-padding its
# spectrum to the 2N x 2N grid, C-hat's row k is the Fourier transform of the
# chirp on the upsampled image (Eq. 5, linear), centred on the visibility's
# grid cell.  The grid cell is 1/L (the upsampled image spans the field of view
# L with 2N pixels of L/2N), so the kernel rows are those of `kernel_box` for a
# geometry with field of view L/2, one gridding tap and S = G.
# ----------------------------------------------------------------------------


def paper_geometry(N: int, L: float, chirp_kind: str = "linear") -> Geometry:
    """Kernel geometry of paper mode: the chirp sampled on the upsampled image
    (offsets (P - G/2) L/G), grid cells 1/L, delta gridding."""
    return Geometry(N, L / 2.0, W=1, chirp_kind=chirp_kind)


def _natural(x):
    """Image with pixel offset p - N/2 moved to index (p - N/2) mod N."""
    N = x.shape[0]
    return np.roll(np.asarray(x), (-(N // 2), -(N // 2)), axis=(0, 1))


def paper_spectrum(x, G: int):
    """P F_N x: the unitary spectrum of the N x N image (natural order) placed
    on the G x G grid (frequency k in [-N/2, N/2) at index k mod G), zeros
    elsewhere.  F_G U x equals this for U = F_G^H P F_N (U is an isometry)."""
    N = x.shape[0]
    XN = np.fft.fft2(_natural(x)) / N
    k = np.arange(-(N // 2), N // 2)
    X = np.zeros((G, G), dtype=np.complex128)
    X[np.ix_(k % G, k % G)] = XN[np.ix_(k % N, k % N)]
    return X


def paper_spectrum_adj(X, N: int):
    """(P F_N)^H X: crop the [-N/2, N/2)^2 block, inverse unitary DFT, back to
    pixel order."""
    G = X.shape[0]
    k = np.arange(-(N // 2), N // 2)
    XN = np.zeros((N, N), dtype=np.complex128)
    XN[np.ix_(k % N, k % N)] = X[np.ix_(k % G, k % G)]
    xn = np.fft.ifft2(XN) * N
    return np.roll(xn, (N // 2, N // 2), axis=(0, 1))


def paper_upsample(x, G: int):
    """U x = F_G^H P F_N x in natural order (offset o at index o mod G)."""
    return np.fft.ifft2(paper_spectrum(x, G)) * G


def paper_phi(N: int, Gm, x):
    """Phi' x = C-hat F U x = C-hat P F_N x."""
    return Gm @ paper_spectrum(np.asarray(x, dtype=np.float64), 2 * N).ravel()


def paper_phi_adj(N: int, Gm, y):
    Xt = np.conj(Gm.T @ np.conj(np.asarray(y))).reshape(2 * N, 2 * N)
    return paper_spectrum_adj(Xt, N)


def paper_visibilities_direct(N: int, L: float, x, uvw, chirp_kind: str = "linear"):
    """The definition itself, for pins: y_k = [F_G (c_k . U x)] at the grid
    cell (u_k L, v_k L) mod G, with c_k the chirp on the upsampled image's
    pixels (offset o at l = o L / G, natural order) and F_G unitary."""
    G = 2 * N
    ux = paper_upsample(np.asarray(x, dtype=np.float64), G)
    o = np.arange(G)
    o = np.where(o < G // 2, o, o - G)
    l = o * (L / G)
    y = np.empty(uvw.shape[0], dtype=np.complex128)
    for k in range(uvw.shape[0]):
        u, v, w = uvw[k]
        c = chirp(l[:, None], l[None, :], w, chirp_kind)
        Y = np.fft.fft2(c * ux) / G
        y[k] = Y[int(math.floor(u * L)) % G, int(math.floor(v * L)) % G]
    return y


def visibilities_direct(geo: Geometry, x, uvw):
    """Brute-force discretisation of Eq. 1 (Eq. 3 with the chirp of Eq. 4)
    as a pixel sum, with the 1/G factor of the unitary F:
      y_k = (1/G) sum_{p,q} x_pq C(l_p, m_q; w_k) exp(-2 pi i (u_k l_p + v_k m_q)),
    l_p = (p - N/2) L/N."""
    N = geo.N
    l = (np.arange(N) - N // 2) * geo.dl
    y = np.empty(uvw.shape[0], dtype=np.complex128)
    for k in range(uvw.shape[0]):
        u, v, w = uvw[k]
        c = chirp(l[:, None], l[None, :], w, geo.chirp_kind)
        ph = np.exp(-2j * np.pi * (u * l[:, None] + v * l[None, :]))
        y[k] = np.sum(np.asarray(x) * c * ph) / geo.G
    return y


def visibilities_direct_dde(geo: Geometry, x, uvw, screens, screen_id):
    """visibilities_direct with a direction-dependent screen per visibility:
      y_k = (1/G) sum_{p,q} x_pq A_k(l_p, m_q) C(l_p, m_q; w_k) exp(-2 pi i (u_k l_p + v_k m_q)),
    A_k = screens[screen_id[k]] read at the image's pixels (index p + N/2)."""
    N = geo.N
    l = (np.arange(N) - N // 2) * geo.dl
    pix = np.arange(N) + N // 2
    y = np.empty(uvw.shape[0], dtype=np.complex128)
    for k in range(uvw.shape[0]):
        u, v, w = uvw[k]
        A = np.asarray(screens[int(screen_id[k])])[np.ix_(pix, pix)]
        c = chirp(l[:, None], l[None, :], w, geo.chirp_kind)
        ph = np.exp(-2j * np.pi * (u * l[:, None] + v * l[None, :]))
        y[k] = np.sum(np.asarray(x) * A * c * ph) / geo.G
    return y


def nufft_type2_direct(geo: Geometry, x, uv):
    """Plain KB-interpolated type-2 NUFFT (no w): y_k = sum_t kb kb X[j0 + t],
    X = F Z A x.  Used to pin the w = 0 case."""
    X = F(geo, AZ(geo, x))
    y = np.empty(uv.shape[0], dtype=np.complex128)
    for k in range(uv.shape[0]):
        gu, gv = uv[k, 0] / geo.du, uv[k, 1] / geo.du
        j0u, j0v = math.floor(gu), math.floor(gv)
        tu = tap_weights(gu - j0u, geo.W, geo.beta)
        tv = tap_weights(gv - j0v, geo.W, geo.beta)
        acc = 0.0j
        for a_, ta in enumerate(taps(geo.W)):
            for b_, tb in enumerate(taps(geo.W)):
                acc += tu[a_] * tv[b_] * X[(j0u + ta) % geo.G, (j0v + tb) % geo.G]
        y[k] = acc
    return y


# ----------------------------------------------------------------------------
# BPDN by Douglas-Rachford (Section 2.3, Eq. 7), Psi = Dirac, real image
# ----------------------------------------------------------------------------


def soft(a, gamma):
    """Proximal operator of gamma ||.||_1 (soft threshold)."""
    return np.sign(a) * np.maximum(np.abs(a) - gamma, 0.0)


def power_norm2(apply, apply_adj, N: int, iters: int = 100):
    """||Phi||^2 of the real-image operator by power iteration on Re Phi^H Phi,
    starting from the unit impulse at the image centre (its spectrum is flat, so
    no row of Phi is orthogonal to it; the constant image has only the zero
    frequency and is annihilated by on-grid sampling at w = 0 that misses it)."""
    x = np.zeros((N, N))
    x[N // 2, N // 2] = 1.0
    lam = 0.0
    for _ in range(iters):
        z = np.real(apply_adj(apply(x)))
        lam = float(np.sqrt(np.sum(z * z)))
        x = z / lam
    return lam


def epsilon_chi2(sigma_n: float, M: int) -> float:
    """eps = sigma_n sqrt(M + 2 sqrt(M)) (chi^2 bound; the paper refers to a
    residual noise level estimator, Section 2.3)."""
    return sigma_n * math.sqrt(M + 2.0 * math.sqrt(M))


def solve_bpdn(apply, apply_adj, y, eps: float, N: int, iters: int,
               inner_iters: int = 10, gamma_frac: float = 1e-2, lam: float = 1.0,
               phi_norm2: float | None = None, power_iters: int = 100,
               history: list | None = None):
    """min ||x||_1 s.t. ||y - Phi x||_2 <= eps over real images x (Eq. 7, Dirac
    basis), by Douglas-Rachford splitting:

      x_t     = P_B(z_t)                         (projection onto the ball)
      z_{t+1} = z_t + lam (soft(2 x_t - z_t, gamma) - x_t)

    with z_0 = Re Phi^H y and gamma = gamma_frac * max|Re Phi^H y|.  P_B is
    computed by dual forward-backward with step mu = 1/||Phi||^2 and a fixed
    number of inner iterations, the dual variable u warm-started across outer
    iterations:
      x = z - Re Phi^H u;  d = u/mu + Phi x - y;
      u <- max(0, 1 - eps/||d||) mu d.
    Returns the last x_t."""
    if phi_norm2 is None:
        phi_norm2 = power_norm2(apply, apply_adj, N, power_iters)
    mu = 1.0 / phi_norm2
    y = np.asarray(y, dtype=np.complex128)
    z = np.real(apply_adj(y))
    gamma = gamma_frac * float(np.max(np.abs(z)))
    u = np.zeros_like(y)
    x = z
    for t in range(iters):
        for _ in range(inner_iters):
            x = z - np.real(apply_adj(u))
            d = u / mu + apply(x) - y
            nd = float(np.sqrt(np.sum(np.abs(d) ** 2)))
            scale = max(0.0, 1.0 - eps / nd) if nd > 0 else 0.0
            u = scale * mu * d
        x = z - np.real(apply_adj(u))
        z = z + lam * (soft(2.0 * x - z, gamma) - x)
        if history is not None:
            history.append(x.copy())
    return x, {"phi_norm2": phi_norm2, "gamma": gamma, "mu": mu}


def snr_db(x, x_rec) -> float:
    """SNR_out = 20 log10(std(x) / std(x - x_rec)) (Section 4.1)."""
    return 20.0 * math.log10(float(np.std(x)) / float(np.std(np.asarray(x) - np.asarray(x_rec))))


def bpdn_closed_form_isometry(ztrue, eps: float, c0: float):
    """For an isometry Phi (Phi^H Phi = I) and real x, ||y - Phi x||^2 =
    c0 + ||b - x||^2 with b = Re Phi^H y, so the BPDN solution is soft(b, l*)
    with ||b - soft(b, l*)||^2 = eps^2 - c0; l* found by bisection."""
    b = np.asarray(ztrue)
    r2 = eps * eps - c0
    if r2 <= 0:
        return b.copy()
    lo, hi = 0.0, float(np.max(np.abs(b)))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        dev = np.sum((b - soft(b, mid)) ** 2)
        if dev > r2:
            hi = mid
        else:
            lo = mid
    return soft(b, lo)
