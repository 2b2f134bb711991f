"""FP64 CPU reference of the surrogate network (test infrastructure only).

Only the tests may import it.  It writes out the network's definition
directly with numpy, channels-last, zero padding:

    h_{-1} = (Re psi, Im psi, |psi|^2 Re psi, |psi|^2 Im psi)
    z_l[p, co] = b_l[co] + sum_{t, ci} W_l[co, t, ci] h_{l-1}[p + d_l o_t, ci]
    h_l = z_l * sigmoid(z_l)                       (l < L-1)
    psi_out = psi_in + z_{L-1}[.., 0] + i z_{L-1}[.., 1]
    loss = mean over all real components of (psi_out - target)^2
           + mass_weight * mean over states of ((M(psi_out) - M(target)) / M(target))^2,
           M(x) = sum over the state's sites of |x|^2
    optional mass projection (inference only): psi_out * sqrt(M_in / M_out)

with o_t = (t // 3 - 1, t % 3 - 1), and its gradient by the chain rule
(backward-data is the transpose convolution with the offsets negated;
silu'(z) = s (1 + z (1 - s)), s = sigmoid(z)).  Parity status: pinned by
central finite differences of the loss (with and without the mass term), the
mass term's closed form on a bias-only network, the forward convolution by
scipy's 2D correlation with the dilated taps, and the mass projection by its
closed form on scaled states (tests/test_surrogate_ref.py).
Parameter layout: per layer W [cout][9][cin] then b [cout].
"""
import numpy as np

N_IN = 4      # input features per pixel


def layer_shapes(channels, layers):
    out = []
    for l in range(layers):
        ci = N_IN if l == 0 else channels
        co = 2 if l == layers - 1 else channels
        out.append((co, ci))
    return out


def unpack(params, channels, layers):
    Ws, bs, off = [], [], 0
    for co, ci in layer_shapes(channels, layers):
        n = co * 9 * ci
        Ws.append(np.asarray(params[off:off + n], dtype=np.float64).reshape(co, 9, ci))
        off += n
        bs.append(np.asarray(params[off:off + co], dtype=np.float64))
        off += co
    return Ws, bs


def shift(x, dy, dx):
    """x[n, y + dy, x + dx, c] with zeros outside the grid."""
    nb, H, Wd, C = x.shape
    out = np.zeros_like(x)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(Wd, Wd - dx)
    if ys < ye and xs < xe:
        out[:, ys:ye, xs:xe, :] = x[:, ys + dy:ye + dy, xs + dx:xe + dx, :]
    return out


def conv(x, Wl, bl, d):
    z = np.zeros(x.shape[:3] + (Wl.shape[0],))
    for t in range(9):
        z += shift(x, d * (t // 3 - 1), d * (t % 3 - 1)) @ Wl[:, t, :].T
    return z + bl


def forward(params, psi, channels, layers, dilations):
    """psi: complex [nb, H, W]; returns psi_out and the activations."""
    Ws, bs = unpack(params, channels, layers)
    r = np.abs(psi) ** 2
    h = np.stack([psi.real, psi.imag, r * psi.real, r * psi.imag], axis=-1).astype(np.float64)
    hs, zs = [h], []
    for l in range(layers):
        z = conv(hs[-1], Ws[l], bs[l], dilations[l])
        zs.append(z)
        if l < layers - 1:
            hs.append(z / (1.0 + np.exp(-z)))
    y = zs[-1]
    return psi + y[..., 0] + 1j * y[..., 1], hs, zs


def loss_and_grad(params, psi, target, channels, layers, dilations, mass_weight=0.0):
    Ws, bs = unpack(params, channels, layers)
    out, hs, zs = forward(params, psi, channels, layers, dilations)
    e = np.stack([(out - target).real, (out - target).imag], axis=-1)
    count = e.size
    loss = float(np.sum(e * e) / count)
    dz = 2.0 * e / count                       # d loss / d z_{L-1}
    if mass_weight:
        # the mass term: d/d out of mean_b delta_b^2 is (2 delta_b / nb) (2 out / M_t,b)
        nb = psi.shape[0]
        m_out = np.sum(np.abs(out) ** 2, axis=(1, 2))
        m_t = np.sum(np.abs(target) ** 2, axis=(1, 2))
        delta = (m_out - m_t) / m_t
        loss += float(mass_weight * np.mean(delta * delta))
        coef = mass_weight * 4.0 * delta / (nb * m_t)
        dz = dz + coef[:, None, None, None] * np.stack([out.real, out.imag], axis=-1)
    grads = [None] * layers
    for l in range(layers - 1, -1, -1):
        x, d = hs[l], dilations[l]
        dW = np.zeros_like(Ws[l])
        for t in range(9):
            xs = shift(x, d * (t // 3 - 1), d * (t % 3 - 1))
            dW[:, t, :] = np.einsum("nyxo,nyxi->oi", dz, xs)
        db = dz.sum(axis=(0, 1, 2))
        grads[l] = (dW, db)
        if l > 0:
            dx = np.zeros(x.shape)
            for t in range(9):
                dx += shift(dz, -d * (t // 3 - 1), -d * (t % 3 - 1)) @ Ws[l][:, t, :]
            z = zs[l - 1]
            sg = 1.0 / (1.0 + np.exp(-z))
            dz = dx * sg * (1.0 + z * (1.0 - sg))
    flat = []
    for dW, db in grads:
        flat.append(dW.ravel())
        flat.append(db)
    return loss, np.concatenate(flat)


def project_mass(psi_in, psi_out):
    """Rescale each state of psi_out ([nb, H, W]) to the mass sum |psi|^2 of
    the matching psi_in state (the NLSE conserves mass)."""
    a = np.sum(np.abs(psi_in) ** 2, axis=(1, 2))
    b = np.sum(np.abs(psi_out) ** 2, axis=(1, 2))
    r = np.where(b > 0, np.sqrt(a / np.where(b > 0, b, 1.0)), 1.0)
    return psi_out * r[:, None, None]
