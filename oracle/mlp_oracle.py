"""Plain FP64 CPU oracle of the learned pose proposal.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the benchmark's CPU-baseline leg may import it; the library never does.  It
shares no code with the CUDA path.

The paper registers from the identity and relies on the adaptive tree to
widen the basin (Sec. 4).  The learned proposal is this project's addition
(no counterpart in the paper): a 3-layer MLP reads the 64 level-1 GMM nodes
(the paper's second level of 8-component GMMs) of both clouds and proposes
an initial pose, which the plain method then refines.  Everything below is
the definition written out in float64:

* Canonical frame of a cloud: the root mean c, the RMS radius
  s = sqrt(trace Sigma_root), and the root eigenvectors V (columns, the
  tree's own convention: descending eigenvalues, largest-|entry| positive,
  the same axes that seed the level-0 children) with the third column
  negated when det V < 0, so that V is a rotation.
* Features of a cloud (64 x 10): level-0 node k sits in group
  k ^ (4 if the third axis was negated), so that the group index is the
  octant of the node's initial mean in the frame; inside a group the live
  children come in order of decreasing weight (ties by index).  A live
  level-0 node whose children all died stands for itself in its group's
  first slot.  Node entry: [64 pi_parent pi_child, V^T (mu - c) / s,
  16 * upper(V^T Sigma V) / s^2] (upper = xx xy xz yy yz zz); empty slots
  are zeros.
* Input x = [features(source), features(target)] (1280), rounded to BF16.
* Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3 with
  BF16 weights (FP32 master copies) and 1280 -> 256 -> 256 -> 9.  The
  default is FP64 throughout; ``act_bf16`` models the stated storage
  precision of the tensor-core path (BF16 hidden activations and BF16
  backward signals into every product) so that the arithmetic of the
  kernels can be checked apart from the effect of that precision.
* Output: y[0:3], y[3:6] are the 6-D rotation representation (Gram-Schmidt
  of two column vectors), y[6:9] the translation, both in canonical
  coordinates: x~_t = R' x~_s + t' with x~ = V^T (x - c) / s per cloud, so
  R' = V_t^T R V_s and t' = V_t^T (R c_s + t - c_t) / s_t for the pose
  x_t = R x_s + t that maps the source into the target.
* Loss per pair: ||R^ - R'||_F^2 + w_t ||t^ - t'||^2, averaged over the batch.
* Optimiser: Adam (bias-corrected first and second moments).

Pins: ``tests/test_oracle_mlp.py`` checks the analytic gradients against
central finite differences, Gram-Schmidt against rotations it must return
unchanged, the first Adam step against its closed form, the features of an
exactly rotated tree against the sign-flip permutation they must undergo,
and the label encoding of such a pair against the flip matrix itself.
"""
from __future__ import annotations

import numpy as np

from oracle import hgmm_oracle as H

IN = 1280
HID = 256
OUT = 9
NODES = 64
PER_NODE = 10
SHAPES = (("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (OUT, HID)), ("b3", (OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
PI_SCALE = 64.0
COV_SCALE = 16.0


# --------------------------------------------------------------------------
# BF16 storage format: round-to-nearest-even of the upper 16 bits of FP32
# --------------------------------------------------------------------------
def bf16(x):
    """Values of x after conversion to bfloat16 (round to nearest, ties to
    even), returned as float64.  Finite inputs only."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[k:k + n].reshape(shape)
        k += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


# --------------------------------------------------------------------------
# Network
# --------------------------------------------------------------------------
def forward(params, X, round_weights=True, act_bf16=False):
    """y (B, 9) for inputs X (B, 1280).  With round_weights the weight
    matrices take their BF16 values (biases stay FP32).  With act_bf16 the
    hidden activations are stored in BF16 before the next product, as the
    tensor-core path stores them."""
    P = unpack(params)
    W = {k: (bf16(P[k]) if round_weights else P[k]) for k in ("W1", "W2", "W3")}
    r = bf16 if act_bf16 else (lambda a: a)
    X = np.asarray(X, np.float64)
    z1 = X @ W["W1"].T + P["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W["W2"].T + P["b2"]
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ W["W3"].T + P["b3"]
    return y, {"X": X, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "W": W}


def gram_schmidt(a1, a2):
    """Rotation with columns b1 = a1/|a1|, b2 = the part of a2 orthogonal to
    b1, normalised, and b3 = b1 x b2.  Works on (..., 3) stacks."""
    b1 = a1 / np.linalg.norm(a1, axis=-1, keepdims=True)
    u = a2 - np.sum(b1 * a2, axis=-1, keepdims=True) * b1
    b2 = u / np.linalg.norm(u, axis=-1, keepdims=True)
    b3 = np.cross(b1, b2)
    return np.stack([b1, b2, b3], axis=-1)


def loss(y, labels, w_t):
    """Mean over the batch of ||GS(y) - R'||_F^2 + w_t ||y_t - t'||^2;
    labels (B, 12) = R' row-major, t'."""
    y = np.asarray(y, np.float64)
    L = np.asarray(labels, np.float64)
    R = gram_schmidt(y[:, 0:3], y[:, 3:6])
    Rs = L[:, :9].reshape(-1, 3, 3)
    e = np.sum((R - Rs) ** 2, axis=(1, 2)) + w_t * np.sum((y[:, 6:9] - L[:, 9:12]) ** 2, axis=1)
    return float(e.mean())


def loss_grad(y, labels, w_t):
    """dL/dy (B, 9) of ``loss``: chain rule through b3 = b1 x b2, the
    normalisations and the projection of a2, written out per column."""
    y = np.asarray(y, np.float64)
    L = np.asarray(labels, np.float64)
    B = y.shape[0]
    a1, a2 = y[:, 0:3], y[:, 3:6]
    n1 = np.linalg.norm(a1, axis=1, keepdims=True)
    b1 = a1 / n1
    d = np.sum(b1 * a2, axis=1, keepdims=True)
    u = a2 - d * b1
    n2 = np.linalg.norm(u, axis=1, keepdims=True)
    b2 = u / n2
    b3 = np.cross(b1, b2)
    Rs = L[:, :9].reshape(-1, 3, 3)
    G1 = 2.0 * (b1 - Rs[:, :, 0])
    G2 = 2.0 * (b2 - Rs[:, :, 1])
    G3 = 2.0 * (b3 - Rs[:, :, 2])
    # b3 = b1 x b2:  d(G3 . b3) = (b2 x G3) . db1 + (G3 x b1) . db2
    gb1 = G1 + np.cross(b2, G3)
    gb2 = G2 + np.cross(G3, b1)
    # b2 = u / |u|
    gu = (gb2 - np.sum(gb2 * b2, axis=1, keepdims=True) * b2) / n2
    # u = a2 - (b1 . a2) b1
    ga2 = gu - np.sum(gu * b1, axis=1, keepdims=True) * b1
    gb1 = gb1 - np.sum(gu * b1, axis=1, keepdims=True) * a2 - d * gu
    # b1 = a1 / |a1|
    ga1 = (gb1 - np.sum(gb1 * b1, axis=1, keepdims=True) * b1) / n1
    gt = 2.0 * w_t * (y[:, 6:9] - L[:, 9:12])
    return np.concatenate([ga1, ga2, gt], axis=1) / B


def backward(params, X, labels, w_t, round_weights=True, act_bf16=False):
    """Loss and its gradient with respect to the FP32 master parameters (the
    BF16 rounding of the weights passes gradients through unchanged).  With
    act_bf16 the forward stores hidden activations in BF16 and the backward
    signals dL/dy, dL/dz2, dL/dz1 that enter a product are stored in BF16 too
    (the bias gradient of the last layer sums the unrounded dL/dy)."""
    y, c = forward(params, X, round_weights, act_bf16)
    r = bf16 if act_bf16 else (lambda a: a)
    dy = loss_grad(y, labels, w_t)
    dyr = r(dy)
    W = c["W"]
    g = {"W3": dyr.T @ c["h2"], "b3": dy.sum(axis=0)}
    dz2 = r((dyr @ W["W3"]) * (c["z2"] > 0))
    g["W2"], g["b2"] = dz2.T @ c["h1"], dz2.sum(axis=0)
    dz1 = r((dz2 @ W["W2"]) * (c["z1"] > 0))
    g["W1"], g["b1"] = dz1.T @ c["X"], dz1.sum(axis=0)
    return loss(y, labels, w_t), pack(g), y


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of every parameter; returns the
    new parameters and moments."""
    m = beta1 * m + (1.0 - beta1) * grads
    v = beta2 * v + (1.0 - beta2) * grads * grads
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------
# Features and the canonical frame
# --------------------------------------------------------------------------
def frame(root_mu, root_Sigma):
    """(c, s, V, flipped): canonical frame of a cloud from its root Gaussian."""
    lam, V = H.sym_eig(np.asarray(root_Sigma, np.float64))
    V = V.copy()
    flipped = bool(np.linalg.det(V) < 0)
    if flipped:
        V[:, 2] = -V[:, 2]
    s = float(np.sqrt(np.maximum(lam, 0.0).sum()))
    return np.asarray(root_mu, np.float64), (s if s > 0 else 1.0), V, flipped


def frame_vector(c, s, V, flipped):
    """16 numbers: c (3), s, V row-major (9), flipped, 0, 0."""
    return np.concatenate([c, [s], V.reshape(-1), [1.0 if flipped else 0.0, 0.0, 0.0]])


def _upper(S):
    return np.array([S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]])


def features(levels, root_mu, root_Sigma):
    """(640 features, 16-number frame) of one cloud from its tree levels 0
    and 1 (objects with pi, mu, Sigma, live)."""
    c, s, V, flipped = frame(root_mu, root_Sigma)
    l0, l1 = levels[0], levels[1]
    F = np.zeros((NODES, PER_NODE))

    def entry(w, mu, S):
        return np.concatenate([[PI_SCALE * w], V.T @ (mu - c) / s,
                               COV_SCALE * _upper(V.T @ S @ V) / (s * s)])

    for k in range(8):
        if not l0.live[k]:
            continue
        group = k ^ (4 if flipped else 0)
        kids = [j for j in range(8) if l1.live[8 * k + j]]
        if not kids:
            F[8 * group] = entry(l0.pi[k], l0.mu[k], l0.Sigma[k])
            continue
        kids.sort(key=lambda j: (-l1.pi[8 * k + j], j))
        for r, j in enumerate(kids):
            g = 8 * k + j
            F[8 * group + r] = entry(l0.pi[k] * l1.pi[g], l1.mu[g], l1.Sigma[g])
    return F.reshape(-1), frame_vector(c, s, V, flipped)


def _unframe(f):
    f = np.asarray(f, np.float64)
    return f[0:3], f[3], f[4:13].reshape(3, 3)


def encode_label(T, frame_src, frame_tgt):
    """12 numbers (R' row-major, t') of the pose T (4x4, source -> target)
    in the two canonical frames."""
    cs, _, Vs = _unframe(frame_src)
    ct, st, Vt = _unframe(frame_tgt)
    R, t = np.asarray(T, np.float64)[:3, :3], np.asarray(T, np.float64)[:3, 3]
    Rp = Vt.T @ R @ Vs
    tp = Vt.T @ (R @ cs + t - ct) / st
    return np.concatenate([Rp.reshape(-1), tp])


def decode(y, frame_src, frame_tgt):
    """Pose T (4x4, source -> target) from one network output y (9)."""
    cs, _, Vs = _unframe(frame_src)
    ct, st, Vt = _unframe(frame_tgt)
    y = np.asarray(y, np.float64)
    Rp = gram_schmidt(y[0:3], y[3:6])
    R = Vt @ Rp @ Vs.T
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = ct + st * (Vt @ y[6:9]) - R @ cs
    return T
