"""Oracle: the learned proposal's network, tables, loss and gradient in FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

Definition restated (the paper has no learned component; this is the
library's extension):
  * state T = set of lines not yet ordered; features x(T) = 16 indicator
    bits, |T|/M, 1 (zero-padded to 32);
  * h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
    o = W4 h3 + b4 (widths 64, 64, 64, 16); weights used in BF16;
  * P(j | T) = softmax_{j in T}( ln wplain(T\\j) + 3 tanh(o_j(T)/3) ),
    Deg_theta(T) = Deg(T) exp(0.7 tanh(o_15(T)/0.7));
  * ln q_theta(z) = sum_l ln P(j_l | S_l) + sum_{l>=1} [ln Deg_theta(S_l)
    + Deg_theta(S_l) ln t_l] - sum ln z;
  * loss = -sum_i w_i ln q_theta(z_i) / sum_i w_i (the -sum ln z term,
    independent of the network, is left out).
Sampling with the trained network (learned_points): the defensive mixture
q = (1 - beta) q_theta + beta g.  With u_0 < beta the plain density g is
drawn (its component pick taken from u_0 / beta; the sector walk divides
log2 u by Deg), otherwise the learned walk: remove from T the first j in T
(ascending) whose cumulative P(j'|T) over j' <= j exceeds the uniform (the
last j in T if none does), then t = u^(1/Deg_theta(T without j)).  Uniforms:
philox.uniforms_fine.  The density is log2 q = log2((1 - beta) q_theta +
beta g), g from sampler.log2_density.

Gradients by explicit backpropagation in float64; pinned by central finite
differences of the loss itself.  forward()/loss_and_grad() round weights,
activations and the backward signals to BF16 at the points where the
device kernels do (FP32 accumulation there, float64 here);
grad_unrounded()/loss_only() use unrounded float64 throughout.  Pins of the
learned sampler: E_g[q/g] = 1 (q is a density on the simplex) and the
zero-output identity.
"""
import numpy as np

IN, HID, OUT = 32, 64, 16
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
         ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (OUT, HID)), ("b4", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)
LAM, KAP = 3.0, 0.7


def bf16(x):
    """Round float64/float32 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    out, k = {}, 0
    for name, shp in SIZES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[k:k + n], dtype=np.float64).reshape(shp)
        k += n
    return out


def features(M):
    S = 1 << M
    X = np.zeros((S, IN))
    T = np.arange(S)
    for k in range(min(M, 16)):
        X[:, k] = (T >> k) & 1
    X[:, 16] = np.array([bin(t).count("1") for t in range(S)]) / M
    X[:, 17] = 1.0
    return X


def forward(params, M):
    """Forward pass as the device runs it: BF16 weights and features, each
    hidden activation rounded to BF16 after bias and ReLU, outputs kept."""
    w = unpack(params)
    W = {k: (bf16(v) if k.startswith("W") else np.asarray(v, dtype=np.float32).astype(np.float64))
         for k, v in w.items()}
    X = bf16(features(M))
    z1 = X @ W["W1"].T + W["b1"]; h1 = bf16(np.maximum(z1, 0))
    z2 = h1 @ W["W2"].T + W["b2"]; h2 = bf16(np.maximum(z2, 0))
    z3 = h2 @ W["W3"].T + W["b3"]; h3 = bf16(np.maximum(z3, 0))
    o = h3 @ W["W4"].T + W["b4"]
    return dict(W=W, X=X, h1=h1, h2=h2, h3=h3, o=o)


def tables(o, deg, wplain, M):
    S = 1 << M
    full = S - 1
    logp = np.full((S, 16), -np.inf)
    for T in range(S):
        js = [j for j in range(M) if T >> j & 1]
        if len(js) < 2:
            continue
        l = np.array([np.log(wplain[T ^ (1 << j)]) + LAM * np.tanh(o[T, j] / LAM) for j in js])
        lse = l.max() + np.log(np.sum(np.exp(l - l.max())))
        for j, lj in zip(js, l):
            logp[T, j] = lj - lse
    degt = np.ones(S)
    for T in range(1, full):
        degt[T] = deg[T] * np.exp(KAP * np.tanh(o[T, 15] / KAP))
    return logp, degt


def loss_and_grad(params, deg, wplain, order, lt, w, M):
    """Loss and d loss / d params (float64), for samples given as descending
    line order (n, >= M) and ln t at levels 1..M-1 (n, >= M)."""
    f = forward(params, M)
    o = f["o"]
    logp, degt = tables(o, deg, wplain, M)
    S = 1 << M
    full = S - 1
    wn = np.asarray(w, dtype=np.float64) / np.sum(w)
    dl = np.zeros((S, 16))      # d loss / d l(T, j)  and  d loss / d ln Deg_theta(T) in column 15
    loss = 0.0
    for i in range(len(wn)):
        if wn[i] == 0:
            continue
        T = full
        lq = 0.0
        for l in range(M - 1):
            j = int(order[i, l])
            lq += logp[T, j]
            for jj in range(M):
                if T >> jj & 1:
                    dl[T, jj] -= wn[i] * ((1.0 if jj == j else 0.0) - np.exp(logp[T, jj]))
            T ^= 1 << j
            lnt = float(lt[i, l + 1])
            lq += np.log(degt[T]) + degt[T] * lnt
            dl[T, 15] -= wn[i] * (1.0 + degt[T] * lnt)
        loss -= wn[i] * lq
    dO = np.zeros_like(o)
    dO[:, :15] = dl[:, :15] * (1 - np.tanh(o[:, :15] / LAM) ** 2)
    dO[:, 15] = dl[:, 15] * (1 - np.tanh(o[:, 15] / KAP) ** 2)
    # backward as the device runs it: the output signal and every hidden
    # signal rounded to BF16 before they enter a product
    dO = bf16(dO)
    W = f["W"]
    g = {}
    g["W4"] = dO.T @ f["h3"]; g["b4"] = dO.sum(0)
    d3 = bf16((dO @ W["W4"]) * (f["h3"] > 0))
    g["W3"] = d3.T @ f["h2"]; g["b3"] = d3.sum(0)
    d2 = bf16((d3 @ W["W3"]) * (f["h2"] > 0))
    g["W2"] = d2.T @ f["h1"]; g["b2"] = d2.sum(0)
    d1 = bf16((d2 @ W["W2"]) * (f["h1"] > 0))
    g["W1"] = d1.T @ f["X"]; g["b1"] = d1.sum(0)
    grad = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return loss, grad, logp, degt


def loss_only(params, deg, wplain, order, lt, w, M, round_weights=False):
    """Loss with unrounded float64 weights (for finite differences)."""
    wts = unpack(params)
    X = features(M)
    h1 = np.maximum(X @ wts["W1"].T + wts["b1"], 0)
    h2 = np.maximum(h1 @ wts["W2"].T + wts["b2"], 0)
    h3 = np.maximum(h2 @ wts["W3"].T + wts["b3"], 0)
    o = h3 @ wts["W4"].T + wts["b4"]
    logp, degt = tables(o, deg, wplain, M)
    wn = np.asarray(w) / np.sum(w)
    full = (1 << M) - 1
    loss = 0.0
    for i in range(len(wn)):
        T = full
        lq = 0.0
        for l in range(M - 1):
            j = int(order[i, l])
            lq += logp[T, j]
            T ^= 1 << j
            lq += np.log(degt[T]) + degt[T] * float(lt[i, l + 1])
        loss -= wn[i] * lq
    return loss


def grad_unrounded(params, deg, wplain, order, lt, w, M):
    """Backpropagation with unrounded float64 weights and features."""
    wts = unpack(params)
    X = features(M)
    z1 = X @ wts["W1"].T + wts["b1"]; h1 = np.maximum(z1, 0)
    z2 = h1 @ wts["W2"].T + wts["b2"]; h2 = np.maximum(z2, 0)
    z3 = h2 @ wts["W3"].T + wts["b3"]; h3 = np.maximum(z3, 0)
    o = h3 @ wts["W4"].T + wts["b4"]
    logp, degt = tables(o, deg, wplain, M)
    S = 1 << M
    full = S - 1
    wn = np.asarray(w) / np.sum(w)
    dl = np.zeros((S, 16))
    for i in range(len(wn)):
        T = full
        for l in range(M - 1):
            j = int(order[i, l])
            for jj in range(M):
                if T >> jj & 1:
                    dl[T, jj] -= wn[i] * ((1.0 if jj == j else 0.0) - np.exp(logp[T, jj]))
            T ^= 1 << j
            dl[T, 15] -= wn[i] * (1.0 + degt[T] * float(lt[i, l + 1]))
    dO = np.zeros_like(o)
    dO[:, :15] = dl[:, :15] * (1 - np.tanh(o[:, :15] / LAM) ** 2)
    dO[:, 15] = dl[:, 15] * (1 - np.tanh(o[:, 15] / KAP) ** 2)
    g = {"W4": dO.T @ h3, "b4": dO.sum(0)}
    d3 = (dO @ wts["W4"]) * (z3 > 0); g["W3"] = d3.T @ h2; g["b3"] = d3.sum(0)
    d2 = (d3 @ wts["W3"]) * (z2 > 0); g["W2"] = d2.T @ h1; g["b2"] = d2.sum(0)
    d1 = (d2 @ wts["W2"]) * (z1 > 0); g["W1"] = d1.T @ X; g["b1"] = d1.sum(0)
    return np.concatenate([g[name].ravel() for name, _ in SIZES])


def learned_points(dens, o, beta, u):
    """Draw from the defensive mixture (1 - beta) q_theta + beta g of one
    graph with network outputs o (2^M x 16, as exported by the library) and
    uniforms u (S x 2M, philox.uniforms_fine).  Returns (z, log2 q, plain)
    with plain = True where the plain density was drawn."""
    from .sampler import log2_density
    M = dens.M
    full = (1 << M) - 1
    deg1, phi1 = dens.deg[0], dens.phi[0]
    wplain = np.ones(1 << M)
    wplain[1:-1] = phi1[1:-1] / deg1[1:-1]
    logp, degt = tables(o, deg1, wplain, M)
    P = np.where(np.isfinite(logp), np.exp(logp), 0.0)
    Pc = np.cumsum(P, axis=1)          # cumulative over j' <= j, in the order of j
    S = u.shape[0]
    lz = np.zeros((S, M))
    plain = u[:, 0] < beta
    for s in range(S):
        T = full
        cur = 0.0
        if plain[s]:
            pick = u[s, 0] / beta
            c1, c3, c4 = dens.C
            comp = 0 if pick < c1 else 1 if pick < c1 + dens.C2 else 2 if pick < c1 + dens.C2 + c3 else 3
            if comp == 1:
                lz[s] = np.log2(-np.log2(u[s, 1:1 + M]))
                continue
            k = 0 if comp == 0 else comp - 1
            deg, phi = dens.deg[k], dens.phi[k]
            for l in range(M - 1):
                target = u[s, 1 + 2 * l] * phi[T]
                acc = 0.0
                chosen = -1
                last = 0
                for j in range(M):
                    if T >> j & 1:
                        acc = acc + phi[T ^ (1 << j)] / deg[T ^ (1 << j)]
                        if chosen < 0 and target < acc:
                            chosen = j
                        last = j
                chosen = last if chosen < 0 else chosen
                lz[s, chosen] = cur
                T ^= 1 << chosen
                cur = cur + np.log2(u[s, 2 + 2 * l]) / deg[T]
        else:
            for l in range(M - 1):
                uc = u[s, 1 + 2 * l]
                js = [j for j in range(M) if T >> j & 1]
                chosen = js[-1]
                for j in js:
                    if uc < Pc[T, j]:
                        chosen = j
                        break
                lz[s, chosen] = cur
                T ^= 1 << chosen
                cur = cur + np.log2(u[s, 2 + 2 * l]) / degt[T]
        lz[s, int(np.log2(T))] = cur
    e = np.exp2(lz)
    ssum = e.sum(1)
    z = e / ssum[:, None]
    lz = lz - np.log2(ssum)[:, None]
    return z, log2_mixture(dens, logp, degt, beta, lz), plain


def log2_learned(logp, degt, lz, M):
    """log2 q_theta at points given by log2 z (S x M): the ordering's
    probabilities times prod Deg_theta(S_l) t_l^Deg_theta(S_l) / prod z."""
    order = np.argsort(-lz, axis=1, kind="stable")
    full = (1 << M) - 1
    out = np.empty(lz.shape[0])
    for s in range(lz.shape[0]):
        T = full
        lq = 0.0
        for l in range(M - 1):
            j = order[s, l]
            lq += logp[T, j] / np.log(2.0)
            T ^= 1 << j
            lq += np.log2(degt[T]) + degt[T] * (lz[s, order[s, l + 1]] - lz[s, j])
        out[s] = lq - lz[s].sum()
    return out


def log2_mixture(dens, logp, degt, beta, lz):
    """log2((1 - beta) q_theta + beta g) at points given by log2 z."""
    from .sampler import log2_density
    a = np.log2(beta) + log2_density(dens, lz)
    b = np.log2(1.0 - beta) + log2_learned(logp, degt, lz, dens.M) if beta < 1 else np.full(lz.shape[0], -np.inf)
    m = np.maximum(a, b)
    return m + np.log2(np.exp2(a - m) + np.exp2(b - m))
