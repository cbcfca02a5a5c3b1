"""HFSO minimax design of the transition samples V(r) (Sec. III-B, III-C, III-E of the paper).

The filter of the hot path takes V as an input. This module finds V for a specification, on the
CPU in FP64: the design is off the hot path and runs once per specification (a bandwidth change
re-indexes V and computes nothing, Sec. III-E).

The design problem (eq. (minimax)): for given L and N, find V(0..L_V-1) and delta that
    minimize delta  subject to  |E_n(w, b)| <= delta
for w in the passband [0, b - Delta/2] and the stopband [b + Delta/2, pi], every band b of the
range and every output phase n = 0..M-1 of the OLS block. E_n = H_n - H_d (eq. (err_min)) is the
error of the time-invariant response H_n that output phase n sees (the PTVIR view of OLS, Sec.
II) against the desired linear-phase response (eq. (OLS_Hnd)).

The responses. Output phase n of a block (output sample mM + n) is the circular convolution of
the block with h = IDFT(H) (eq. (OLS_dn)) read at position O + n. Tap q reaches the input sample
q positions back when q <= n + O, and, through the circular wrap, the sample N - q positions
ahead otherwise. So H_n(w) = sum_{q <= n+O} h(q) e^{-jwq} + sum_{q > n+O} h(q) e^{-jw(q-N)}. The
last phase n = M - 1 has no wrapped tap: its response is the DTFT of h, the response d_{M-1} of
eq. (OLS_dn). The desired response is e^{-jwD} on the passband and 0 on the stopband, D = (L-1)/2,
in the alignment of this library (O samples of history precede the stream; the paper's H_d
carries M - 1 more samples of delay in its alignment, a common factor that leaves |E_n| unchanged).

h is affine in V through the cosine form of d_{M-1}(q, b) (Sec. III-B), so each E_n(w, b) is an
affine complex function of V. |E| <= delta is convex (a second-order cone). It is solved here as
a sequence of linear programs: each adds, for the points where the current solution violates the
bound most, the supporting half-plane Re(e^{-j theta} E) <= delta with theta = arg E; the LP
bound then converges to the minimax modulus (cutting planes). The solver is scipy's HiGHS.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def order_estimate(delta_p: float, delta_s: float, Delta: float) -> float:
    """Initial filter order N_D of eq. (filt_order_estim): -4 pi log10(10 dp ds) / (3 Delta)."""
    return -4.0 * math.pi * math.log10(10.0 * delta_p * delta_s) / (3.0 * Delta)


def choose_N(L: int) -> int:
    """N = 0.9 L log2(L) rounded to the nearest power of two (Sec. III-D)."""
    n_hat = 0.9 * L * math.log2(L)
    q = round(math.log2(n_hat))
    return 1 << q


def band_bins(bN: int, Delta_N: int) -> tuple[int, int]:
    """(k1, k2) of eq. (k_var) for the transition centre b_N: k1 = b_N - Delta_N/2 + 1,
    k2 = b_N + Delta_N/2 - 1."""
    return bN - Delta_N // 2 + 1, bN + Delta_N // 2 - 1


def h_basis(N: int, L: int, k1: int, LV: int) -> np.ndarray:
    """h(q) = c_0(q) + sum_r V(r) c_{r+1}(q), the cosine form of d_{M-1}(q, b) (Sec. III-B).
    Returns C with shape (N, L_V + 1): column 0 is the fixed part (DC and passband bins), column
    r + 1 the coefficient of V(r)."""
    q = np.arange(N, dtype=np.float64)
    D = (L - 1) / 2.0
    C = np.zeros((N, LV + 1))
    C[:, 0] = 1.0
    for k in range(1, k1):
        C[:, 0] += 2.0 * np.cos(2.0 * np.pi * k * (q - D) / N)
    for r in range(LV):
        C[:, r + 1] = 2.0 * np.cos(2.0 * np.pi * (k1 + r) * (q - D) / N)
    return C / N


def phase_responses(C: np.ndarray, N: int, L: int, omega: np.ndarray) -> np.ndarray:
    """F[n, i, j] = sum_q C[q, j] e^{-j w_i (s_n(q) - D)}: the responses of the OLS output phases
    n = 0..M-1 (taps q <= n + O at delay q, later taps wrapped to delay q - N), each column of C
    taken as h, with the desired delay D = (L-1)/2 removed."""
    O = L - 1
    M = N - O
    D = O / 2.0
    q = np.arange(N)
    E = np.exp(-1j * np.outer(omega, q - D))              # (K, N)
    P = np.cumsum(E[:, :, None] * C[None, :, :], axis=1)  # (K, N, J): sum over q' <= q
    total = P[:, -1, :]
    wrap = np.exp(1j * omega * N)[:, None]                # delay q - N for the wrapped taps
    out = np.empty((M, len(omega), C.shape[1]), dtype=np.complex128)
    for n in range(M):
        head = P[:, n + O, :]
        out[n] = head + wrap * (total - head)
    return out


def grid(bN: int, Delta_N: int, N: int, K: int) -> tuple[np.ndarray, np.ndarray]:
    """K points over the passband [0, b - Delta/2] and stopband [b + Delta/2, pi] of band b_N, in
    proportion to their widths; returns (w, 1 for passband points else 0)."""
    wc = (bN - Delta_N / 2) * 2 * np.pi / N
    ws = (bN + Delta_N / 2) * 2 * np.pi / N
    Kp = max(2, int(round(K * wc / (wc + np.pi - ws))))
    Ks = max(2, K - Kp)
    w = np.concatenate([np.linspace(0.0, wc, Kp), np.linspace(ws, np.pi, Ks)])
    d = np.concatenate([np.ones(Kp), np.zeros(Ks)])
    return w, d


@dataclass
class Design:
    V: np.ndarray          # L_V transition samples
    delta: float           # max |E_n(w, b)| over the grid, every band and phase
    N: int
    L: int
    M: int
    Delta_N: int
    bN: tuple[int, int]
    iterations: int


def error_system(N: int, L: int, Delta_N: int, bN_lo: int, bN_hi: int, K: int):
    """(A, c) with E = A V + c for every (band, phase, grid point), flattened: A is
    (points, L_V) complex, c (points,) complex."""
    LV = Delta_N - 1
    As, cs = [], []
    for bN in range(bN_lo, bN_hi + 1):
        k1, k2 = band_bins(bN, Delta_N)
        if k1 < 1 or k2 > N // 2 - 2:
            raise ValueError(f"b_N={bN} outside the range eq. (k_var) allows for N={N}")
        w, d = grid(bN, Delta_N, N, K)
        F = phase_responses(h_basis(N, L, k1, LV), N, L, w)   # (M, K, LV + 1)
        As.append(F[:, :, 1:].reshape(-1, LV))
        cs.append((F[:, :, 0] - d[None, :]).reshape(-1))
    return np.concatenate(As), np.concatenate(cs)


def design_transition(N: int, L: int, Delta_N: int, bN_lo: int, bN_hi: int, K: int = 1000,
                      tol: float = 1e-3, max_iter: int = 500, init_stride: int = 1000,
                      cuts: int = 500) -> Design:
    """Minimax V for one (N, L): eq. (minimax) over b_N in [bN_lo, bN_hi], every output phase and
    K grid points per band (cutting-plane LP on the complex modulus). Stops when the largest
    modulus on the full grid is within `tol` (relative) of the LP's bound."""
    from scipy.optimize import linprog
    LV = Delta_N - 1
    A, c = error_system(N, L, Delta_N, bN_lo, bN_hi, K)
    npts = len(c)
    # start: a sparse subset of points, eight half-planes each
    idx = np.arange(0, npts, init_stride)
    thetas = np.arange(8) * (np.pi / 4)
    rows_A, rows_b = [], []

    def add(points, th):
        e = np.exp(-1j * th)
        rows_A.append(np.hstack([(e[:, None] * A[points]).real, -np.ones((len(points), 1))]))
        rows_b.append(-(e * c[points]).real)

    for t in thetas:
        add(idx, np.full(len(idx), t))
    cost = np.zeros(LV + 1)
    cost[-1] = 1.0
    bounds = [(None, None)] * LV + [(0, None)]
    V = np.zeros(LV)
    it = 0
    for it in range(1, max_iter + 1):
        A_ub, b_ub = np.vstack(rows_A), np.concatenate(rows_b)
        res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs")
        if res.status != 0:
            raise RuntimeError(f"LP failed: {res.message}")
        V, lp_delta = res.x[:LV], res.x[-1]
        E = A @ V + c
        mag = np.abs(E)
        worst = mag.max()
        if worst <= lp_delta * (1 + tol) + 1e-15:
            break
        if it % 5 == 0:
            # drop half-planes far from binding (slack above half the bound); the LP stays small
            keep = (b_ub - A_ub @ res.x) < 0.5 * lp_delta
            rows_A, rows_b = [A_ub[keep]], [b_ub[keep]]
        # the most violated points get the half-plane through their current error direction
        viol = np.nonzero(mag > lp_delta * (1 + tol))[0]
        take = viol[np.argsort(mag[viol])[::-1][:cuts]]
        add(take, np.angle(E[take]))
    E = A @ V + c
    return Design(V=V, delta=float(np.abs(E).max()), N=N, L=L, M=N - L + 1, Delta_N=Delta_N,
                  bN=(bN_lo, bN_hi), iterations=it)


def candidate_rows(N: int, L: int, LV: int, k1: np.ndarray, n: np.ndarray, omega: np.ndarray,
                   d: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(A, c) with E = A V + c for a list of (band k1, output phase n, frequency w, desired d)
    points, in FP64: the rows of eq. (minimax) at those points only (same responses as
    phase_responses). A is (P, L_V) complex, c (P,) complex."""
    O = L - 1
    D = O / 2.0
    q = np.arange(N)
    P = len(k1)
    A = np.empty((P, LV), dtype=np.complex128)
    c = np.empty(P, dtype=np.complex128)
    for kk in np.unique(k1):
        sel = np.nonzero(k1 == kk)[0]
        C = h_basis(N, L, int(kk), LV)                                   # (N, L_V + 1)
        s = np.where(q[None, :] <= n[sel, None] + O, q[None, :], q[None, :] - N)
        F = np.exp(-1j * omega[sel, None] * (s - D)) @ C                 # (p, L_V + 1)
        A[sel] = F[:, 1:]
        c[sel] = F[:, 0] - d[sel]
    return A, c


def design_transition_gpu(N: int, L: int, Delta_N: int, bN_lo: int, bN_hi: int, K: int = 1000,
                          tol: float = 1e-3, max_iter: int = 500, cuts: int = 500,
                          check: int = 4000) -> Design:
    """eq. (minimax) as design_transition, with the search over (band, phase, frequency) on the GPU.

    Each round, the kernel behind vbw_ptvir_error evaluates max_n |E_n(w, b)| at every grid point
    of every band for the current V (float32, within about 1e-7 x sum |h| of the exact value) and
    returns the phase reaching it. The `check` largest points are then re-evaluated in FP64 on the
    host (candidate_rows) and the violated ones give the LP's new half-planes, as in
    design_transition. Stops when the FP64 maximum over those points is within `tol` (relative)
    of the LP's bound; the returned delta is that FP64 maximum. No matrix over every point is
    formed, so the grid size is bounded by device memory, not by host memory."""
    import torch
    from scipy.optimize import linprog

    from . import vbw

    LV = Delta_N - 1
    O = L - 1
    bNs = list(range(bN_lo, bN_hi + 1))
    k1s = []
    ws, ds = [], []
    for bN in bNs:
        k1, k2 = band_bins(bN, Delta_N)
        if k1 < 1 or k2 > N // 2 - 2:
            raise ValueError(f"b_N={bN} outside the range eq. (k_var) allows for N={N}")
        w, d = grid(bN, Delta_N, N, K)
        k1s.append(k1)
        ws.append(w)
        ds.append(d)
    Kmax = max(len(w) for w in ws)
    # rows of equal length: a short row repeats its last point (evaluated twice, harmless)
    W = np.stack([np.concatenate([w, np.full(Kmax - len(w), w[-1])]) for w in ws])
    Dd = np.stack([np.concatenate([d, np.full(Kmax - len(d), d[-1])]) for d in ds])
    dev = torch.device("cuda")
    t_bands = torch.tensor(np.asarray(k1s, np.int32), device=dev)
    t_w = torch.tensor(W, dtype=torch.float64, device=dev)
    t_d = torch.tensor(Dd.astype(np.float32), device=dev)
    t_err = torch.empty(W.shape, dtype=torch.float32, device=dev)
    t_ph = torch.empty(W.shape, dtype=torch.int32, device=dev)
    k1_arr = np.asarray(k1s)

    def worst_points(V):
        plan = vbw.Plan(N, O, V)
        try:
            vbw.vbw_ptvir_error(plan.handle, t_bands, t_w, t_d, t_err, t_ph)
            torch.cuda.synchronize()
        finally:
            plan.close()
        err = t_err.cpu().numpy().ravel()
        top = np.argpartition(err, -min(check, err.size))[-min(check, err.size):]
        r, col = np.divmod(top, Kmax)
        n = t_ph.cpu().numpy().ravel()[top]
        A, c = candidate_rows(N, L, LV, k1_arr[r], n, W[r, col], Dd[r, col])
        return A, c

    rows_A, rows_b = [], []

    def add(A, c, th):
        e = np.exp(-1j * th)
        rows_A.append(np.hstack([(e[:, None] * A).real, -np.ones((len(c), 1))]))
        rows_b.append(-(e * c).real)

    # start: the worst points of a linear transition, eight half-planes each
    V = np.linspace(1.0, 0.0, LV + 2)[1:-1]
    A, c = worst_points(V)
    take = np.argsort(np.abs(A @ V + c))[::-1][:cuts]
    for t in np.arange(8) * (np.pi / 4):
        add(A[take], c[take], np.full(len(take), t))
    cost = np.zeros(LV + 1)
    cost[-1] = 1.0
    bounds = [(None, None)] * LV + [(0, None)]
    it = 0
    worst = np.inf
    for it in range(1, max_iter + 1):
        A_ub, b_ub = np.vstack(rows_A), np.concatenate(rows_b)
        res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs")
        if res.status != 0:
            raise RuntimeError(f"LP failed: {res.message}")
        V, lp_delta = res.x[:LV], res.x[-1]
        A, c = worst_points(V)
        E = A @ V + c
        mag = np.abs(E)
        worst = mag.max()
        if worst <= lp_delta * (1 + tol) + 1e-15:
            break
        if it % 5 == 0:
            keep = (b_ub - A_ub @ res.x) < 0.5 * lp_delta
            rows_A, rows_b = [A_ub[keep]], [b_ub[keep]]
        viol = np.nonzero(mag > lp_delta * (1 + tol))[0]
        take = viol[np.argsort(mag[viol])[::-1][:cuts]]
        add(A[take], c[take], np.angle(E[take]))
    return Design(V=V, delta=float(worst), N=N, L=L, M=N - L + 1, Delta_N=Delta_N,
                  bN=(bN_lo, bN_hi), iterations=it)


def design_procedure(Delta: float, delta_E: float, b_lo: float, b_hi: float, K: int = 1000,
                     delta_p: float | None = None, delta_s: float | None = None):
    """The design procedure of Sec. III-D: estimate N_D (eq. (filt_order_estim)) and N, solve
    eq. (minimax), then lower N_D while delta <= delta_E (raising it while delta > delta_E). The
    band range [b_lo, b_hi] and Delta are in radians; Delta and b are discretized to bins of
    2 pi / N. Returns the design with the smallest L that meets delta_E."""
    dp = delta_p if delta_p is not None else delta_E
    ds = delta_s if delta_s is not None else delta_E
    ND = int(math.ceil(order_estimate(dp, ds, Delta)))
    if ND % 2:
        ND += 1   # even order: integer delay (L - 1)/2
    best = None
    tried = set()
    while ND not in tried and ND >= 2:
        tried.add(ND)
        L = ND + 1
        N = choose_N(L)
        Delta_N = int(round(Delta * N / (2 * math.pi)))
        bN_lo = int(round(b_lo * N / (2 * math.pi)))   # b discretized to bins (printed b values
        bN_hi = int(round(b_hi * N / (2 * math.pi)))   # are rounded, e.g. 0.8594 pi = 55 bins of 128)
        d = design_transition(N, L, Delta_N, bN_lo, bN_hi, K)
        if d.delta <= delta_E:
            best = d
            ND -= 2
        else:
            if best is not None:
                break
            ND += 2
    if best is None:
        raise RuntimeError("no order met the specification")
    return best
