"""CPU oracle of the learned weight proposal and its training (FP64, numpy).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests, the
smoke check and bench.py's CPU-baseline leg use it; the CUDA library never
does.

The paper solves the moment conditions (Eqs. momcondmv, cond_two,
cond_alpha) for non-negative weights with a linear program (Sec. 4.1).  The
learned path proposes the weights with a small network instead and keeps
only proposals that, after an exact correction, satisfy the same conditions
and signs; everything else goes to the LP.  The pieces:

* features(): the neighbourhood N_i (annulus of Eq. neighbourhood) as K = 32
  slots ordered by (45-degree segment of Sec. 4.2, squared distance, index),
  with the scaled offsets xi = (x_j - x_i)/h of Eq. momcondmv and a mask;
  input row [xi_x(32), xi_y(32), mask(32)].  The order and xi are float32
  quantities from float32 positions (the network's input precision).
* forward()/backward(): the network 96 -> 256 -> 256 -> 256 -> 32 with GELU
  (the tanh form) after each hidden layer; W_l is [out x in].
* loss(): mean squared error over the valid slots against the LP weights
  f~ of the same particle (f~ = h^2 f, Eq. momcondmv scaling).
* adamw(): Adam with decoupled weight decay (Loshchilov and Hutter).
* learned_stencil(): the candidates are the slots holding the small
  neighbourhood of Sec. 4.3 (the closest particle of every segment: the
  columns the LP itself works on), ranked by the network's proposal (larger
  first, ties to the lower slot).  The proposal chooses the stencil's
  support: five candidates at a time, in the order subset_order() fixes
  (increasing sum of ranks, ties lexicographic: the top five first), the
  moment conditions V_S f = b (rows (1,0) (0,1) (2,0) (1,1) (0,2) of Eq.
  momcondmv, b from Eqs. cond_two, cond_alpha) are solved on the support S.
  The first support whose solution is non-negative (Sec. 3.1) with residual
  |V_S f - b|_inf <= 1e-12 is the stencil: the projection of the proposal
  onto the moment conditions within its support, an exact vertex of the same
  feasible set the LP searches.  Each support is screened first in binary32
  (square_solve32: every operation rounded to float32, the same sequence as
  the GPU's), and only a support whose binary32 weights all exceed -1e-6 is
  solved in FP64 (square_solve) and tested; FP64 weights in [-1e-13, 0) are
  zeros of the vertex; at most MAX_SOLVES = 4 supports reach the FP64
  solve.  No passing support: the particle goes to the LP.
* support(), project(), gram_ok(): the least-change correction
      f_S = f0_S + V_S^T (V_S V_S^T)^{-1} (b - V_S f0_S)
  of a proposal on a support of up to eight slots (the smallest change that
  meets the moment conditions), with its conditioning test; reference
  pieces for the square solve (on five slots the two coincide).
"""
import itertools

import numpy as np

K_SLOTS = 32
N_IN = 3 * K_SLOTS
HIDDEN = 256
N_OUT = K_SLOTS
SHAPES = ((HIDDEN, N_IN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (N_OUT, HIDDEN))
N_PARAMS = sum(o * i + o for o, i in SHAPES)  # 164,640
SUPPORT_MAX = 8
ACCEPT_RESID = 1e-12
B_RHS = np.array([0.0, 0.0, 2.0, 0.0, 2.0])  # rows (1,0) (0,1) (2,0) (1,1) (0,2)


# -- parameter vector ------------------------------------------------------------
def unflatten(theta):
    """Flat vector [W1, b1, W2, b2, W3, b3, W4, b4] -> list of (W, b)."""
    out, o = [], 0
    for rows, cols in SHAPES:
        W = theta[o:o + rows * cols].reshape(rows, cols)
        o += rows * cols
        b = theta[o:o + rows]
        o += rows
        out.append((W, b))
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


# -- bf16 rounding (round to nearest even on the float32 bit pattern) ---------------
def to_bf16(a):
    """Round to bfloat16 (returned as float64 holding the bf16 value): first
    to float32, then the upper 16 bits with round-to-nearest-even."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


# -- features ----------------------------------------------------------------------
def segment(dx, dy):
    """45-degree segment of an offset (Sec. 4.2): half-open angular sectors
    [k pi/4, (k+1) pi/4) counter-clockwise from +x, decided exactly."""
    if dx > 0 and 0 <= dy < dx:
        return 0
    if dx > 0 and dy >= dx:
        return 1
    if dx <= 0 and dy > -dx:
        return 2
    if dx < 0 and 0 < dy <= -dx:
        return 3
    if dx < 0 and 0 >= dy > dx:
        return 4
    if dx < 0 and dy <= dx:
        return 5
    if dx >= 0 and -dy > dx:
        return 6
    return 7


def features(x, y, h, i, row):
    """Input row (bf16 values) and slot -> particle map (-1 = empty) of
    particle i whose neighbourhood is `row` (indices, any order).  All float32:
    positions rounded to float32, dx = x_j - x_i, the squared distance d2 and
    xi = dx * (1/h) (products and sums rounded separately, 1/h computed in
    FP64 and rounded to float32).  Slots are ordered by the 32-bit key
    segment * 2^28 + (bit pattern of d2) / 8 (the 3 lowest mantissa bits
    dropped), then by index."""
    f32 = np.float32
    inv_h = f32(1.0 / h)
    ent = []
    for j in row:
        j = int(j)
        dx = f32(f32(x[j]) - f32(x[i]))
        dy = f32(f32(y[j]) - f32(y[i]))
        d2 = f32(f32(dx * dx) + f32(dy * dy))
        key = (segment(dx, dy) << 28) | (int(np.array(d2, dtype=np.float32).view(np.uint32)) >> 3)
        ent.append((key, j, dx, dy))
    ent.sort(key=lambda e: (e[0], e[1]))
    X = np.zeros(N_IN)
    slots = np.full(K_SLOTS, -1, dtype=np.int64)
    for k, (_, j, dx, dy) in enumerate(ent[:K_SLOTS]):
        X[k] = f32(dx * inv_h)
        X[K_SLOTS + k] = f32(dy * inv_h)
        X[2 * K_SLOTS + k] = 1.0
        slots[k] = j
    return to_bf16(X), slots


# -- network -------------------------------------------------------------------------
GELU_C = np.sqrt(2.0 / np.pi)
GELU_A = 0.044715


def gelu(z):
    """GELU in its tanh form: 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def forward(theta, X, bf16_acts=False):
    """Rows of X [B, 96] -> proposals [B, 32].  bf16_acts rounds the hidden
    activations to bf16 between layers (the precision the GPU keeps them
    in).  Returns (Y, cache)."""
    layers = unflatten(theta)
    a = np.asarray(X, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        cache.append((a, z))
        if l < len(layers) - 1:
            a = gelu(z)
            if bf16_acts:
                a = to_bf16(a)
        else:
            a = z
    return a, cache


def loss(Y, T, M):
    """Mean of M (Y - T)^2 over the valid slots, and dL/dY."""
    cnt = max(float(np.sum(M)), 1.0)
    d = (Y - T) * M
    return float(np.sum(d * d) / cnt), 2.0 * d / cnt


def backward(theta, cache, dY):
    """Gradient of sum(dY * Y) with respect to theta (flat, same layout)."""
    layers = unflatten(theta)
    grads = [None] * len(layers)
    g = dY
    for l in range(len(layers) - 1, -1, -1):
        a, z = cache[l]
        if l < len(layers) - 1:
            g = g * gelu_grad(z)
        W, _ = layers[l]
        grads[l] = (g.T @ a, g.sum(axis=0))
        g = g @ W
    return flatten(grads)


def adamw(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One AdamW step (t counts from 1); returns (theta', m', v')."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + weight_decay * theta)
    return theta, m, v


# -- projection onto the moment conditions ---------------------------------------------
def vandermonde(xi, eta):
    """Rows (1,0) (0,1) (2,0) (1,1) (0,2) of Eq. momcondmv at the given columns."""
    xi = np.asarray(xi, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    return np.stack([xi, eta, xi * xi, xi * eta, eta * eta])


def support(f0, slots, cap=SUPPORT_MAX, allowed=None):
    """Slots of the support: the (up to) cap valid slots (holding a particle
    of `allowed`, if given) with the largest positive proposal, ties to the
    lower slot, returned in slot order.  The comparisons are made on the
    float32 proposals."""
    f0 = np.asarray(f0, dtype=np.float32)
    ok = set(int(a) for a in allowed if a >= 0) if allowed is not None else None
    cand = [k for k in range(len(f0)) if slots[k] >= 0 and f0[k] > 0 and (ok is None or int(slots[k]) in ok)]
    cand.sort(key=lambda k: (-float(f0[k]), k))
    return sorted(cand[:cap])


def project(xi, eta, f0, b=B_RHS):
    """Least-change correction of f0 onto V f = b; returns (f, residual)."""
    V = vandermonde(xi, eta)
    f0 = np.asarray(f0, dtype=np.float64)
    r = b - V @ f0
    f = f0 + V.T @ np.linalg.solve(V @ V.T, r)
    return f, float(np.max(np.abs(V @ f - b)))


def gram_ok(V, rel=1e-10):
    """Cholesky of G = V V^T written out; False if a pivot is at most rel
    times the largest diagonal entry (the rows are then nearly dependent)."""
    G = V @ V.T
    n = G.shape[0]
    L = np.zeros_like(G)
    gmax = float(np.max(np.diag(G)))
    for a in range(n):
        d = G[a, a] - float(np.sum(L[a, :a] ** 2))
        if not d > rel * gmax:
            return False
        L[a, a] = np.sqrt(d)
        for q in range(a + 1, n):
            L[q, a] = (G[q, a] - float(np.sum(L[q, :a] * L[a, :a]))) / L[a, a]
    return True




def square_solve(V, b, rel=1e-12):
    """Solution of the 5 x 5 system V f = b by Gaussian elimination with
    partial pivoting (first largest |pivot| in the column, full row swaps),
    or None when a pivot is at most rel times the largest |entry| of V."""
    A = np.array(V, dtype=np.float64)
    r = np.array(b, dtype=np.float64)
    n = A.shape[0]
    vmax = float(np.max(np.abs(A)))
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if not abs(A[p, k]) > rel * vmax:
            return None
        if p != k:
            A[[k, p]] = A[[p, k]]
            r[[k, p]] = r[[p, k]]
        for q in range(k + 1, n):
            m = A[q, k] / A[k, k]
            A[q, k:] = A[q, k:] - m * A[k, k:]
            r[q] = r[q] - m * r[k]
    f = np.zeros(n)
    for k in range(n - 1, -1, -1):
        f[k] = (r[k] - float(np.dot(A[k, k + 1:], f[k + 1:]))) / A[k, k]
    return f


SCREEN_TOL = np.float32(1e-6)  # binary32 screen: weights above -SCREEN_TOL go to the FP64 solve
SCREEN_PIVOT = np.float32(1e-6)  # binary32 screen: relative pivot threshold
SNAP = 1e-13  # FP64 weights in [-SNAP, 0) are zeros of the vertex
MAX_SOLVES = 4  # FP64 solves per particle at most (supports that passed the screen)


def subset_order(nc):
    """The 5-subsets of candidate ranks 0..nc-1 in the order they are tried:
    increasing sum of ranks, ties in lexicographic order (the network's top
    five first, then one rank swapped in at a time, and so on)."""
    return sorted(itertools.combinations(range(nc), 5), key=lambda r: (sum(r), r))


def square_solve32(xi, eta):
    """Binary32 Gaussian elimination of V_S f = b on five columns, every
    product, reciprocal and difference rounded to float32 in this order:
    V entries xi, eta, xi*xi, xi*eta, eta*eta from float32(xi), float32(eta);
    pivot = first largest |entry| of the column at or below the diagonal,
    None if it is not above SCREEN_PIVOT * (largest |V entry|); rcp_k =
    1 / A[k][k] (one rounding); rows below get A[q][c] - (A[q][k] rcp_k) *
    A[k][c] for c > k and the right-hand side alike; back substitution
    f_k = (r_k - sum_q A[k][q] f_q) * rcp_k with the sum taken
    q = k+1, ..., 4."""
    f32 = np.float32
    A = []
    for r in range(5):
        A.append([f32(0)] * 6)
    for c in range(5):
        a, e = f32(xi[c]), f32(eta[c])
        col = (a, e, f32(a * a), f32(a * e), f32(e * e))
        for r in range(5):
            A[r][c] = col[r]
    for r in range(5):
        A[r][5] = f32(2.0) if r in (2, 4) else f32(0.0)
    vmax = f32(0.0)
    for r in range(5):
        for c in range(5):
            vmax = max(vmax, abs(A[r][c]))
    tiny = f32(SCREEN_PIVOT * vmax)
    rcp = [f32(0.0)] * 5
    for k in range(5):
        p = k
        for q in range(k + 1, 5):
            if abs(A[q][k]) > abs(A[p][k]):
                p = q
        if not abs(A[p][k]) > tiny:
            return None
        A[k], A[p] = A[p], A[k]
        rcp[k] = f32(f32(1.0) / A[k][k])
        for q in range(k + 1, 5):
            m = f32(A[q][k] * rcp[k])
            for c in range(k + 1, 6):
                A[q][c] = f32(A[q][c] - f32(m * A[k][c]))
    f = [f32(0.0)] * 5
    for k in range(4, -1, -1):
        acc = A[k][5]
        for q in range(k + 1, 5):
            acc = f32(acc - f32(A[k][q] * f[q]))
        f[k] = f32(acc * rcp[k])
    return np.array(f, dtype=np.float32)


def candidates(f0, slots, small=None, cap=SUPPORT_MAX):
    """Candidate slots ranked by proposal (larger first, ties to the lower
    slot): the slots holding a small-neighbourhood particle (small: its 8
    indices, -1 empty), or, without small, the cap best valid slots."""
    p32 = np.asarray(f0, dtype=np.float32)
    ok = set(int(a) for a in small if a >= 0) if small is not None else None
    c = [k for k in range(len(p32)) if slots[k] >= 0 and (ok is None or int(slots[k]) in ok)]
    c.sort(key=lambda k: (-float(p32[k]), k))
    return c[:cap]


def learned_stencil(x, y, h, i, slots, f0, small=None, trials=False):
    """The learned stencil of particle i from its slot map, proposal and
    small neighbourhood (8 indices, -1 empty; None: the 8 best valid slots
    are the candidates): (accepted, particle indices, f~, f~_ii), the nonzero
    weights in slot order; with trials=True also the number of supports
    screened."""
    ranked = candidates(f0, slots, small)
    inv_h = 1.0 / h
    tried = solves = 0
    for sub in subset_order(len(ranked)):
        tried += 1
        S = sorted(ranked[r] for r in sub)
        js = [int(slots[k]) for k in S]
        xi = np.array([(x[j] - x[i]) * inv_h for j in js])
        eta = np.array([(y[j] - y[i]) * inv_h for j in js])
        f32 = square_solve32(xi, eta)
        if f32 is None or not np.all(f32 >= -SCREEN_TOL):
            continue
        solves += 1
        V = vandermonde(xi, eta)
        f = square_solve(V, B_RHS)
        if f is not None:
            f = np.where((f < 0.0) & (f >= -SNAP), 0.0, f)
            if np.all(f >= 0.0) and float(np.max(np.abs(V @ f - B_RHS))) <= ACCEPT_RESID:
                nz = [q for q in range(5) if f[q] != 0.0]
                fo = f[nz]
                out = (True, [js[q] for q in nz], fo, -float(np.sum(fo)))
                return out + (tried,) if trials else out
        if solves == MAX_SOLVES:
            break
    out = (False, [], None, 0.0)
    return out + (tried,) if trials else out
