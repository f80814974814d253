"""An independent composition of the Radar-STDA network from PyTorch
float64 library operators (conv2d, conv_transpose2d, batch_norm, conv1d,
sigmoid), used as a pin of the oracle's forward pass and, through PyTorch
autograd, of its gradient."""
import numpy as np
import torch
import torch.nn.functional as F

from paper_2307_09063_gb300 import inputs as I


def torch_reference(params, buffers, x, requires_grad=False):
    """The same network composed from PyTorch float64 library operators.
    params / buffers: float32 numpy blobs; x: [3][H][W] numpy or a float64
    tensor. Returns (z [H][W], block outputs) as tensors when requires_grad,
    else as numpy arrays."""
    out, blocks, _ = torch_forward(params, buffers, x, requires_grad)
    if requires_grad:
        return out, blocks
    return out.detach().numpy(), [b.detach().numpy() for b in blocks]


def torch_forward(params, buffers, x, requires_grad=False, bn_training=False, stats=None):
    """x [frames][H][W] (one window) or [B][frames][H][W] (a batch). With
    bn_training every BN normalises with its input's batch statistics
    (appended to `stats` as (mean, biased var) when given)."""
    batched = np.ndim(x) == 4
    frames = int(np.shape(x)[1 if batched else 0])  # stacked maps (3 in the paper; 2 or 4 in the fusion variants)
    P = {k: torch.tensor(params[o:o + s].astype(np.float64), requires_grad=requires_grad)
         for k, (o, s) in I.param_offsets(frames).items()}
    bufs, off = {}, 0
    for name, c in I.bn_table():
        bufs[name] = (torch.tensor(buffers[off:off + c].astype(np.float64)),
                      torch.tensor(buffers[off + c:off + 2 * c].astype(np.float64)))
        off += 2 * c

    def bn(t, name):
        if bn_training:
            if stats is not None:
                stats.append((t.mean(dim=(0, 2, 3)), t.var(dim=(0, 2, 3), unbiased=False)))
            return F.batch_norm(t, None, None, P[name + ".gamma"], P[name + ".beta"], training=True, eps=1e-5)
        m, v = bufs[name]
        return F.batch_norm(t, m, v, P[name + ".gamma"], P[name + ".beta"], training=False, eps=1e-5)

    a = x if isinstance(x, torch.Tensor) else torch.tensor(np.asarray(x, np.float64))
    if not batched:
        a = a[None]
    a = F.relu(bn(F.conv2d(a, P["stem.w"].view(8, frames, 3, 3), padding=1), "stem.bn"))
    skips, blocks = [], []
    for b in range(6):
        ci, co, p = I.CIN[b], I._cout(b), f"blk{b}"
        w1, w3 = P[p + ".w1"].view(ci, 1, 1, 1), P[p + ".w3"].view(ci, 1, 3, 3)
        if I.ENC[b]:
            t1, t2 = F.conv2d(a, w1, groups=ci), F.conv2d(a, w3, padding=1, groups=ci)
        else:
            t1, t2 = F.conv_transpose2d(a, w1, groups=ci), F.conv_transpose2d(a, w3, padding=1, groups=ci)
        x1 = F.relu(bn(t1, p + ".bn1") + bn(t2, p + ".bn2") + bn(a, p + ".bn3"))
        if I.ENC[b]:
            main = F.conv2d(x1, P[p + ".w2"].view(co, ci, 3, 3), stride=2, padding=1)
            res = F.conv2d(a, P[p + ".rw"].view(co, ci, 3, 3), P[p + ".rb"], stride=2, padding=1)
        else:
            main = F.conv_transpose2d(x1, P[p + ".w2"].view(ci, co, 4, 4), stride=2, padding=1)
            res = F.conv_transpose2d(a, P[p + ".rw"].view(ci, co, 4, 4), P[p + ".rb"], stride=2, padding=1)
        y = F.relu(bn(main, p + ".bn")) + res
        g = y.mean(dim=(2, 3))
        y = y * torch.sigmoid(F.conv1d(g[:, None, :], P[p + ".eca"].view(1, 1, 3), padding=1))[:, 0, :, None, None]
        if b == 3:
            y = y + skips[1]
        if b == 4:
            y = y + skips[0]
        if b < 2:
            skips.append(y)
        blocks.append(y[0])
        a = y
    out = torch.sigmoid(F.conv2d(a, P["out.w"].view(1, 8, 3, 3), P["out.b"], padding=1))
    return (out[:, 0] if batched else out[0, 0]), blocks, P
