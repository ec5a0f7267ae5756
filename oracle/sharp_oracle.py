"""FP64 CPU oracle for the RAAR hot path of SHARP (arXiv:1602.01448).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this module: it exists so that ``tests/``, the package smoke check
and the CPU-baseline leg of ``bench.py`` can compare the CUDA library against
a plain, slow, obviously correct restatement of the paper.  It shares no code,
table or helper with the CUDA sources.

Everything is complex128 / float64 NumPy, one frame at a time, in the order
the paper states the operators.  ``scipy.fft`` (pocketfft, with its stack of
frames split over the host's cores; ``numpy.fft`` where SciPy is missing)
serves as the 2D DFT library primitive; its convention is pinned in the tests
against a brute-force DFT.

Readings of the paper taken here (each also listed in the design notes):
  R1  RAAR update (Sec. 2.2, reconstruction sequence): the printed operator
      2b P_Q P_a + (1-2b) P_a + b (P_Q - I) does not converge; the update used
      is Luke's RAAR, 2b P_Q P_a + (1-2b) P_a + b (I - P_Q).  The printed form
      stays available as ``form="printed"``.
  R2  DFT sign (Eq. 2): the solver uses the unitary e^{-2 pi i q.r} transform
      and amplitudes a = sqrt(I) on that unitary scale.
  R3  Zero modulus in P_a (Eq. 7): Fz/|Fz| is taken as 1 where |Fz| = 0.
  R4  (Q*Q)^{-1} where the illumination sum D = Q*Q is tiny (Eq. 9): the
      object is 0 where D <= 1e-12 max D.
  R5  Positions are integer top-left corners (Sec. 2.1); ``wrap`` indexes the
      object modulo its size (periodic boundary of Fig. 3).
  R6  Probe update (Eq. 10): where the denominator is <= 1e-12 of its maximum
      the old probe value is kept.
  R7  Metrics (Eqs. 11-14) are ratios of Euclidean norms (not squared); each
      RAAR step reports them for the iterate entering that step; the overlap
      metric of an iterate uses the projector of the probe that formed it;
      eps_Delta of the first step compares with a zero iterate.
  R8  eps_0 (Eq. 14) uses the closed-form optimal global phase.
  R12 Illumination drift (Sec. 2.2 pathologies; sequence step 7): the centre
      of mass is the |w|^2-weighted mean of the frame indices; the frame
      centre is index m/2 per axis; the shift is d = floor(c - m/2 + 1/2)
      and w is rolled by -d (periodic within the frame).  The object follows
      by itself: the next object update uses the shifted probe.
  R13 Illumination Fourier constraints (sequence step 7): F is the unitary
      transform of Eq. 2; a mask multiplies Fw, amplitudes a_w replace |Fw|
      (phase 1 where Fw = 0, as R3).  Order: Eq. 10, constraint, centring.
  R14 Initial illumination (sequence step 2; Sec. 3.2 variant): the average
      frame is the mean over frames of a_i^2 on the unitary scale; its
      square root is inverse-transformed and centred in the frame (rolled
      by m/2, i.e. the spectrum multiplied by (-1)^(qy+qx)).  With a
      threshold t in (0, 1], values below t * max go to 0 and the others to
      the mean of the values at or above it.

Parity is pinned for every function below (see tests/test_oracle_*.py) except
where a docstring says "parity unpinned".
"""
from __future__ import annotations

import os

import numpy as np

try:
    import scipy.fft as _sfft
except ImportError:  # pragma: no cover - both machines have SciPy
    _sfft = None

D_REL_THRESHOLD = 1e-12      # R4
PROBE_REL_THRESHOLD = 1e-12  # R6


# --------------------------------------------------------------------------
# Eq. 2 -- two-dimensional unitary DFT over the last two axes
# --------------------------------------------------------------------------
def fft_workers() -> int:
    """Host threads the library transform may use (all cores)."""
    return (os.cpu_count() or 1) if _sfft is not None else 1


def fft2u(z):
    """F: unitary 2D DFT of each m x m frame (Eq. 2, reading R2)."""
    z = np.asarray(z, dtype=np.complex128)
    if _sfft is not None:
        return _sfft.fft2(z, norm="ortho", workers=fft_workers())
    return np.fft.fft2(z, norm="ortho")


def ifft2u(Z):
    """F*: inverse of ``fft2u`` (adjoint of the unitary DFT)."""
    Z = np.asarray(Z, dtype=np.complex128)
    if _sfft is not None:
        return _sfft.ifft2(Z, norm="ortho", workers=fft_workers())
    return np.fft.ifft2(Z, norm="ortho")


# --------------------------------------------------------------------------
# Sec. 2.1 -- frame extraction T_(i) and illumination operator Q (Eqs. 3-6)
# --------------------------------------------------------------------------
def frame_indices(p, m, shape, wrap=False):
    """Row and column indices of the object pixels r + x_(i) seen by a frame
    with top-left corner p = (row, col) (Sec. 2.1 grid, reading R5)."""
    ny, nx = shape
    r0, c0 = int(p[0]), int(p[1])
    rows = np.arange(r0, r0 + m)
    cols = np.arange(c0, c0 + m)
    if wrap:
        rows %= ny
        cols %= nx
    else:
        if r0 < 0 or c0 < 0 or r0 + m > ny or c0 + m > nx:
            raise ValueError(f"frame at {p} leaves the {ny}x{nx} object; use wrap")
    return rows, cols


def split(psi, w, pos, wrap=False):
    """Q psi: z_(i)(r) = w(r) psi(r + x_(i)) for every frame (Sec. 2.1, Eq. 5)."""
    psi = np.asarray(psi, dtype=np.complex128)
    w = np.asarray(w, dtype=np.complex128)
    m = w.shape[0]
    z = np.empty((len(pos), m, m), dtype=np.complex128)
    for i, p in enumerate(pos):
        rows, cols = frame_indices(p, m, psi.shape, wrap)
        z[i] = w * psi[np.ix_(rows, cols)]
    return z


def overlap(z, w, pos, shape, wrap=False):
    """Q* z = sum_i T_(i)^T (conj(w) z_(i)): adjoint of ``split`` (Eq. 5)."""
    w = np.asarray(w, dtype=np.complex128)
    m = w.shape[0]
    out = np.zeros(shape, dtype=np.complex128)
    for i, p in enumerate(pos):
        rows, cols = frame_indices(p, m, shape, wrap)
        np.add.at(out, np.ix_(rows, cols), np.conj(w) * z[i])
    return out


def illumination(w, pos, shape, wrap=False):
    """D = Q*Q = sum_i T_(i)^T |w|^2, the denominator of Eq. 9 (real image)."""
    w = np.asarray(w, dtype=np.complex128)
    m = w.shape[0]
    out = np.zeros(shape, dtype=np.float64)
    w2 = np.abs(w) ** 2
    for i, p in enumerate(pos):
        rows, cols = frame_indices(p, m, shape, wrap)
        np.add.at(out, np.ix_(rows, cols), w2)
    return out


def object_update(z, w, pos, shape, wrap=False):
    """psi <- Q*z / Q*Q (Eq. 9), 0 where D <= 1e-12 max D (reading R4)."""
    D = illumination(w, pos, shape, wrap)
    num = overlap(z, w, pos, shape, wrap)
    ok = D > D_REL_THRESHOLD * D.max()
    return np.where(ok, num / np.where(ok, D, 1.0), 0.0)


def probe_update(z, psi, pos, w_old, wrap=False):
    """w <- S* diag(T conj(psi)) z / S* T |psi|^2 (Eq. 10): per probe pixel the
    sum over frames of conj(psi patch) * z divided by the sum of |psi patch|^2;
    the old value is kept where that sum is tiny (reading R6)."""
    psi = np.asarray(psi, dtype=np.complex128)
    w_old = np.asarray(w_old, dtype=np.complex128)
    m = w_old.shape[0]
    num = np.zeros((m, m), dtype=np.complex128)
    den = np.zeros((m, m), dtype=np.float64)
    for i, p in enumerate(pos):
        rows, cols = frame_indices(p, m, psi.shape, wrap)
        patch = psi[np.ix_(rows, cols)]
        num += np.conj(patch) * z[i]
        den += np.abs(patch) ** 2
    ok = den > PROBE_REL_THRESHOLD * den.max()
    return np.where(ok, num / np.where(ok, den, 1.0), w_old)


# --------------------------------------------------------------------------
# Sec. 2.2 -- projections (Eqs. 7, 8) and the RAAR update
# --------------------------------------------------------------------------
def data_project(z, a):
    """P_a z = F* (Fz / |Fz|) a (Eq. 7), phase 1 where |Fz| = 0 (reading R3)."""
    Z = fft2u(z)
    mag = np.abs(Z)
    phase = np.where(mag > 0, Z / np.where(mag > 0, mag, 1.0), 1.0)
    return ifft2u(np.asarray(a, dtype=np.float64) * phase)


def overlap_project(z, w, pos, shape, wrap=False):
    """P_Q z = Q (Q*Q)^{-1} Q* z (Eq. 8)."""
    return split(object_update(z, w, pos, shape, wrap), w, pos, wrap)


def raar_update(z, a, w, pos, shape, beta=0.75, wrap=False, form="luke"):
    """One RAAR frame update (Sec. 2.2 reconstruction sequence).

    form="luke"   : 2b P_Q P_a z + (1-2b) P_a z + b (I - P_Q) z   (reading R1)
    form="printed": 2b P_Q P_a z + (1-2b) P_a z + b (P_Q - I) z   (as printed)
    """
    pa = data_project(z, a)
    pq_pa = overlap_project(pa, w, pos, shape, wrap)
    pq_z = overlap_project(z, w, pos, shape, wrap)
    if form == "luke":
        tail = beta * (z - pq_z)
    elif form == "printed":
        tail = beta * (pq_z - z)
    else:
        raise ValueError(form)
    return 2.0 * beta * pq_pa + (1.0 - 2.0 * beta) * pa + tail


# --------------------------------------------------------------------------
# Eqs. 11-14 -- metrics
# --------------------------------------------------------------------------
def norm(x):
    return float(np.sqrt(np.sum(np.abs(np.asarray(x)) ** 2)))


def eps_a(z, a):
    """||(P_a - I) z|| / ||a|| (Eq. 11)."""
    return norm(data_project(z, a) - z) / norm(a)


def eps_q(z, a, w, pos, shape, wrap=False):
    """||(P_Q - I) z|| / ||a|| (Eq. 12)."""
    return norm(overlap_project(z, w, pos, shape, wrap) - z) / norm(a)


def eps_delta(z_new, z_old, a):
    """||z^(l) - z^(l-1)|| / ||a|| (Eq. 13)."""
    return norm(np.asarray(z_new) - np.asarray(z_old)) / norm(a)


def global_phase(u, v):
    """e^{i phi} minimising ||e^{i phi} u - v||: <u,v>/|<u,v>| with
    <u,v> = sum conj(u) v (reading R8); 1 if <u,v> = 0."""
    s = np.vdot(np.asarray(u).ravel(), np.asarray(v).ravel())
    return s / abs(s) if abs(s) > 0 else 1.0 + 0.0j


def eps_0(z, z0, w, pos, shape, wrap=False):
    """min_phi ||Q*(e^{i phi} z - z0)|| / ||Q* z0|| (Eq. 14)."""
    u = overlap(z, w, pos, shape, wrap)
    v = overlap(z0, w, pos, shape, wrap)
    return norm(global_phase(u, v) * u - v) / norm(v)


def eps_0_object(psi, psi_true, w, pos, shape, wrap=False):
    """Eq. 14 evaluated at z = Q psi, z0 = Q psi_true: with D = Q*Q this is
    min_phi ||D (e^{i phi} psi - psi_true)|| / ||D psi_true||."""
    D = illumination(w, pos, shape, wrap)
    u = D * np.asarray(psi, dtype=np.complex128)
    v = D * np.asarray(psi_true, dtype=np.complex128)
    return norm(global_phase(u, v) * u - v) / norm(v)


def object_nrmse(psi, psi_true, w, pos, shape, wrap=False, frac=0.1):
    """Object NRMSE over well-illuminated pixels (D >= frac max D), modulo the
    closed-form global phase (secondary report of reading R8; pinned against
    a hand-written masked sum)."""
    D = illumination(w, pos, shape, wrap)
    sel = D >= frac * D.max()
    u = np.asarray(psi)[sel]
    v = np.asarray(psi_true)[sel]
    return norm(global_phase(u, v) * u - v) / norm(v)


# --------------------------------------------------------------------------
# Amplitude loss and its gradient (differentiable form of Eq. 1)
# --------------------------------------------------------------------------
def amp_loss(psi, w, a, pos, wrap=False):
    """L(psi, w) = sum_i || |F Q(psi, w)_(i)| - a_(i) ||^2."""
    z = split(psi, w, pos, wrap)
    return float(np.sum((np.abs(fft2u(z)) - np.asarray(a, dtype=np.float64)) ** 2))


def amp_loss_grad(psi, w, a, pos, wrap=False):
    """Conjugate (Wirtinger) gradients dL/d conj(psi), dL/d conj(w).

    With r = z - P_a z (unitary F, phase 1 at |Fz| = 0 as in R3):
      dL/d conj(psi) = Q* r                  (adjoint of Eq. 5)
      dL/d conj(w)   = sum_i conj(T_(i) psi) r_(i)   (adjoint of Eq. 6)
    A real perturbation h of psi_k changes L by 2 h Re(g_k) to first order.
    """
    psi = np.asarray(psi, dtype=np.complex128)
    z = split(psi, w, pos, wrap)
    r = z - data_project(z, a)
    g_psi = overlap(r, w, pos, psi.shape, wrap)
    m = np.asarray(w).shape[0]
    g_w = np.zeros((m, m), dtype=np.complex128)
    for i, p in enumerate(pos):
        rows, cols = frame_indices(p, m, psi.shape, wrap)
        g_w += np.conj(psi[np.ix_(rows, cols)]) * r[i]
    return g_psi, g_w


def forward_amplitudes(psi, w, pos, wrap=False):
    """a_(i) = |F w psi(r + x_(i))| (Eq. 1) on the unitary scale."""
    return np.abs(fft2u(split(psi, w, pos, wrap)))


# --------------------------------------------------------------------------
# Reconstruction loop (Sec. 2.2 reconstruction sequence)
# --------------------------------------------------------------------------
# --------------------------------------------------------------------------
# Sec. 2.2 -- illumination pathologies and initialisation (reconstruction
# sequence steps 2 and 7; the threshold variant of Sec. 3.2)
# --------------------------------------------------------------------------
def probe_centroid(w):
    """Centre of mass (row, col) of |w|^2 over frame indices 0..m-1 (R12)."""
    inten = np.abs(np.asarray(w, dtype=np.complex128)) ** 2
    m = inten.shape[0]
    idx = np.arange(m, dtype=np.float64)
    total = inten.sum()
    row = float((inten.sum(axis=1) * idx).sum() / total)
    col = float((inten.sum(axis=0) * idx).sum() / total)
    return row, col


def probe_center(w):
    """Drift correction: roll w within the frame so that the centre of mass
    of |w|^2 moves to the frame centre m/2 (R12).  Returns (w, (dy, dx))."""
    w = np.asarray(w, dtype=np.complex128)
    m = w.shape[0]
    cy, cx = probe_centroid(w)
    dy = int(np.floor(cy - m / 2 + 0.5))
    dx = int(np.floor(cx - m / 2 + 0.5))
    return np.roll(w, (-dy, -dx), axis=(0, 1)), (dy, dx)


def probe_fourier_mask(w, mask):
    """w <- F^-1{(F w) m_w} (sequence step 7, R13)."""
    return ifft2u(fft2u(w) * np.asarray(mask, dtype=np.float64))


def probe_fourier_amplitude(w, a_w):
    """w <- F^-1{(F w)/|F w| a_w} (sequence step 7, R13; phase 1 where Fw = 0)."""
    W = fft2u(w)
    mag = np.abs(W)
    phase = np.where(mag > 0, W / np.where(mag > 0, mag, 1.0), 1.0)
    return ifft2u(np.asarray(a_w, dtype=np.float64) * phase)


def probe_from_mean_frame(a, threshold=0.0):
    """Initial illumination from the average frame (sequence step 2; with a
    threshold, the variant of Sec. 3.2), centred in the frame (R14)."""
    a = np.asarray(a, dtype=np.float64)
    m = a.shape[-1]
    mean = np.mean(a ** 2, axis=0)
    if threshold > 0:
        keep = mean >= threshold * mean.max()
        mean = np.where(keep, mean[keep].mean(), 0.0)
    w = ifft2u(np.sqrt(mean))
    return np.roll(w, (m // 2, m // 2), axis=(0, 1))


def refine_probe(w, probe_mask=None, probe_amp=None, probe_com=False):
    """The steps after Eq. 10 in sequence step 7: the Fourier mask if given,
    else the Fourier amplitudes if given, then the centring (R13, R12)."""
    if probe_mask is not None:
        w = probe_fourier_mask(w, probe_mask)
    elif probe_amp is not None:
        w = probe_fourier_amplitude(w, probe_amp)
    if probe_com:
        w, _ = probe_center(w)
    return w


def raar_reconstruct(a, pos, shape, w0, psi0, n_iter, beta=0.75, probe_every=0,
                     wrap=False, form="luke", psi_true=None, w_true=None,
                     record_metrics=True, probe_mask=None, probe_amp=None, probe_com=False):
    """Run ``n_iter`` RAAR steps from z^(0) = Q psi^(0) with illumination w0.

    Step l (1-based): z^(l) = RAAR(z^(l-1)) with the current probe; then the
    object psi^(l) = Q*z^(l)/Q*Q (Eq. 9); then, when probe_every > 0 and
    l % probe_every == 0, the probe from Eq. 10 using psi^(l) and z^(l),
    followed by the optional Fourier constraint and centring (``refine_probe``).

    Metrics recorded at step l describe z^(l-1), the iterate entering the step
    (reading R7): eps_a, eps_Q (projector of the probe that formed z^(l-1)),
    eps_Delta = ||z^(l-1) - z^(l-2)|| / ||a|| with z^(-1) = 0, and, when
    ``psi_true`` is given, eps_0 of the object psi^(l) (Eq. 14 at z = Q psi).
    Returns dict(psi, w, z, history) with history a list of per-step dicts.
    """
    a = np.asarray(a, dtype=np.float64)
    w = np.asarray(w0, dtype=np.complex128).copy()
    z = split(psi0, w, pos, wrap)
    w_formed = w          # probe that formed the current iterate z
    z_prev = np.zeros_like(z)
    history = []
    psi = np.asarray(psi0, dtype=np.complex128).copy()
    for step in range(1, n_iter + 1):
        rec = {"step": step}
        if record_metrics:
            rec["eps_a"] = eps_a(z, a)
            rec["eps_q"] = eps_q(z, a, w_formed, pos, shape, wrap)
            rec["eps_delta"] = eps_delta(z, z_prev, a)
        z_next = raar_update(z, a, w, pos, shape, beta, wrap, form)
        w_formed = w
        psi = object_update(z_next, w, pos, shape, wrap)
        if probe_every and step % probe_every == 0:
            w = probe_update(z_next, psi, pos, w, wrap)
            w = refine_probe(w, probe_mask, probe_amp, probe_com)
        if psi_true is not None:
            wt = w if w_true is None else w_true
            rec["eps_0"] = eps_0_object(psi, psi_true, wt, pos, shape, wrap)
        z_prev, z = z, z_next
        history.append(rec)
    return {"psi": psi, "w": w, "z": z, "history": history}
