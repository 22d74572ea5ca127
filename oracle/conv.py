"""Float64 reference of the warm-start network's operations (forward and backward).

Test infrastructure only (see the package docstring). The learned GS warm start is not in
the paper: it is an engineering extension that predicts a GS starting phase (the paper's
Section 3 random phase is its fallback). Every operation here is written from its
definition; gradients are pinned against central finite differences in the tests.

Layout: activations [B, H, W, C] (channels last); conv weights [Cout, 3, 3, Cin]; 3x3
convolution with zero padding 1 and stride 1 (cross-correlation, as in the GPU kernels).
"""

import numpy as np


def conv3x3(x, w, b=None):
    """y[b,y,x,o] = sum_{ky,kx,i} x[b, y+ky-1, x+kx-1, i] * w[o, ky, kx, i] (+ bias[o])."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, H, W, Ci = x.shape
    Co = w.shape[0]
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((B, H, W, Co))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("bhwi,oi->bhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :], optimize=True)
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3x3_dgrad(dy, w):
    """dL/dx for y = conv3x3(x, w): dx[b,y,x,i] = sum dy[b, y-ky+1, x-kx+1, o] w[o,ky,kx,i]."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    B, H, W, Co = dy.shape
    Ci = w.shape[3]
    dyp = np.zeros((B, H + 2, W + 2, Co))
    dyp[:, 1:-1, 1:-1, :] = dy
    dx = np.zeros((B, H, W, Ci))
    for ky in range(3):
        for kx in range(3):
            # x position p receives dy at p - (ky - 1): in padded coordinates p + 1 - (ky - 1)
            dx += np.einsum("bhwo,oi->bhwi", dyp[:, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W, :], w[:, ky, kx, :], optimize=True)
    return dx


def conv3x3_wgrad(x, dy):
    """dL/dw[o,ky,kx,i] = sum_{b,y,x} dy[b,y,x,o] * x[b, y+ky-1, x+kx-1, i]."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    B, H, W, Ci = x.shape
    Co = dy.shape[3]
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    dw = np.zeros((Co, 3, 3, Ci))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwi->oi", dy, xp[:, ky:ky + H, kx:kx + W, :], optimize=True)
    return dw


def bias_grad(dy):
    return np.asarray(dy, np.float64).sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    x = np.asarray(x, np.float64)
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_bwd(dy):
    dy = np.asarray(dy, np.float64)
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    x = np.asarray(x, np.float64)
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_bwd(dy):
    dy = np.asarray(dy, np.float64)
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def phase_loss(out, z, wts, eps=1e-12):
    """Offset-invariant phase loss per sample, averaged over the batch.

    out [B,H,W,2] = (u, v): predicted phasor y = (u + i v)/|u + i v|; z [B,H,W] complex
    unit label phasors; wts [B,H,W] non-negative pixel weights. For each sample
    S = sum w y conj(z) and L_b = 1 - |S| / sum w; L = mean_b L_b. A global phase offset of
    the prediction (or the label) leaves L unchanged.
    """
    out = np.asarray(out, np.float64)
    u, v = out[..., 0], out[..., 1]
    r = np.sqrt(u * u + v * v) + eps
    y = (u + 1j * v) / r
    S = np.sum(wts * y * np.conj(z), axis=(1, 2))
    Wt = np.sum(wts, axis=(1, 2))
    return float(np.mean(1.0 - np.abs(S) / Wt))


def phase_loss_grad(out, z, wts, eps=1e-12):
    """dL/d(u, v) of phase_loss, written out (chain rule through the normalisation)."""
    out = np.asarray(out, np.float64)
    B = out.shape[0]
    u, v = out[..., 0], out[..., 1]
    r = np.sqrt(u * u + v * v) + eps
    a, bb = u / r, v / r
    c, d = z.real, z.imag
    Sr = np.sum(wts * (a * c + bb * d), axis=(1, 2))
    Si = np.sum(wts * (bb * c - a * d), axis=(1, 2))
    mag = np.sqrt(Sr * Sr + Si * Si) + eps
    Wt = np.sum(wts, axis=(1, 2))
    k = (-1.0 / (B * Wt * mag))[:, None, None]
    ga = k * wts * (Sr[:, None, None] * c - Si[:, None, None] * d)
    gb = k * wts * (Sr[:, None, None] * d + Si[:, None, None] * c)
    r3 = r ** 3
    gu = v * (ga * v - gb * u) / r3
    gv = u * (gb * u - ga * v) / r3
    return np.stack([gu, gv], axis=-1)


def bilinear_resample(x, Ho, Wo):
    """Bilinear resampling of x [H, W] (float64) to Ho x Wo with half-pixel centres.

    Output pixel (oy, ox) is centred at input coordinates
        sy = (oy + 1/2) * H / Ho - 1/2,   sx = (ox + 1/2) * W / Wo - 1/2,
    each clamped to [0, H - 1] and [0, W - 1] (the edge value is held beyond the outer
    pixel centres). With y0 = floor(sy), y1 = min(y0 + 1, H - 1), fy = sy - y0 and the same
    for x, the value is
        (1-fy)(1-fx) x[y0,x0] + (1-fy) fx x[y0,x1] + fy (1-fx) x[y1,x0] + fy fx x[y1,x1].
    At Ho = H, Wo = W every sample falls on an input centre (the identity).
    """
    x = np.asarray(x, np.float64)
    H, W = x.shape

    def axis(n_in, n_out):
        s = np.clip((np.arange(n_out) + 0.5) * n_in / n_out - 0.5, 0.0, n_in - 1.0)
        i0 = np.floor(s).astype(np.int64)
        i1 = np.minimum(i0 + 1, n_in - 1)
        return i0, i1, s - i0

    y0, y1, fy = axis(H, Ho)
    x0, x1, fx = axis(W, Wo)
    fy = fy[:, None]
    fx = fx[None, :]
    return ((1 - fy) * (1 - fx) * x[np.ix_(y0, x0)] + (1 - fy) * fx * x[np.ix_(y0, x1)]
            + fy * (1 - fx) * x[np.ix_(y1, x0)] + fy * fx * x[np.ix_(y1, x1)])


def phase_of_uv(uv, Ho, Wo):
    """The warm start's output phase at Ho x Wo: u and v (channels 0 and 1 of the head
    output uv [H, W, C]) resampled bilinearly (``bilinear_resample``), then
    phase = atan2(v, u) in (-pi, pi]. Resampling the phasor components rather than the
    angle keeps the result continuous across the +-pi cut."""
    uv = np.asarray(uv, np.float64)
    u = bilinear_resample(uv[..., 0], Ho, Wo)
    v = bilinear_resample(uv[..., 1], Ho, Wo)
    return np.arctan2(v, u)


def area_average(target, R):
    """The network input: target [H, W] averaged over disjoint (H/R) x (W/R) blocks to R x R."""
    t = np.asarray(target, np.float64)
    H, W = t.shape
    return t.reshape(R, H // R, R, W // R).mean(axis=(1, 3))


def adam_step(w, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) at time step ``step`` >= 1.

        m <- beta1 m + (1 - beta1) g;   v <- beta2 v + (1 - beta2) g^2
        m_hat = m / (1 - beta1^step);   v_hat = v / (1 - beta2^step)
        w <- w - lr * m_hat / (sqrt(v_hat) + eps)

    Returns the new (w, m, v) as float64 arrays; the inputs are not modified.
    """
    w = np.asarray(w, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return w - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
