"""A float64 PyTorch emulation of the BF16 training path (test infrastructure): the same
forward and backward as the library's tensor-core training kernels, with bf16 rounding at the
same points, so that a GPU result can be compared with the bf16 arithmetic it should have
done rather than only with float64."""
import numpy as np
import torch
import torch.nn.functional as F

import oracle


def _bf16(x):
    return x.to(torch.bfloat16).double()


def bf16_emulation(frames, tgt, spec, wts, gain=1.0, offset=100.0, rounding=True):
    """Loss and gradients of the BF16 training path emulated in float64 PyTorch, rounding to
    bf16 exactly where the library does: every stored activation (the ReLU outputs), the
    weights of layers 1..L-1, and every stored activation gradient dz (pre-activation
    gradients, ReLU mask applied from the bf16 activations).  The first layer, the heads, the
    loss and every accumulation stay at full precision; the loss and its head gradient come
    from the oracle's formula (oracle.loss).  rounding = False drops the roundings: the result
    is then the exact float64 gradient (the structure check of tests/test_bf16_emulation.py)."""
    bf16 = _bf16 if rounding else (lambda x: x)
    dil = spec.dilations
    L = len(dil)
    x0 = torch.from_numpy(((frames.astype(np.float32) - np.float32(offset)) / np.float32(gain)
                           * np.float32(spec.in_scale)).astype(np.float64))[:, None]
    w = [torch.from_numpy(np.asarray(a, dtype=np.float32).astype(np.float64)) for a in wts.conv_w]
    b = [torch.from_numpy(np.asarray(a, dtype=np.float32).astype(np.float64)) for a in wts.conv_b]
    wq = [w[0]] + [bf16(x) for x in w[1:]]
    acts = [bf16(torch.relu(F.conv2d(x0, w[0], b[0], padding=dil[0], dilation=dil[0])))]
    for l in range(1, L):
        acts.append(bf16(torch.relu(F.conv2d(acts[-1], wq[l], b[l], padding=dil[l], dilation=dil[l]))))
    hw = torch.from_numpy(np.asarray(wts.head_w, dtype=np.float32).astype(np.float64))
    hb = torch.from_numpy(np.asarray(wts.head_b, dtype=np.float32).astype(np.float64))
    h = F.conv2d(acts[-1], hw[:, :, None, None], hb)
    val, dh = oracle.loss(h.numpy(), tgt)
    dh = torch.from_numpy(dh)
    dhw = torch.einsum("bkhw,bchw->kc", dh, acts[-1])
    dhb = dh.sum(dim=(0, 2, 3))
    dz = bf16(F.conv_transpose2d(dh, hw[:, :, None, None]) * (acts[-1] > 0))
    dws, dbs = [None] * L, [None] * L
    for l in range(L - 1, 0, -1):
        dws[l] = torch.nn.grad.conv2d_weight(acts[l - 1], w[l].shape, dz, padding=dil[l], dilation=dil[l])
        dbs[l] = dz.sum(dim=(0, 2, 3))
        dz = bf16(F.conv_transpose2d(dz, wq[l], padding=dil[l], dilation=dil[l]) * (acts[l - 1] > 0))
    dws[0] = torch.nn.grad.conv2d_weight(x0, w[0].shape, dz, padding=dil[0], dilation=dil[0])
    dbs[0] = dz.sum(dim=(0, 2, 3))
    return val, [torch.cat([x.reshape(-1) for x in dws]).numpy(), torch.cat([x.reshape(-1) for x in dbs]).numpy(),
                 dhw.reshape(-1).numpy(), dhb.numpy()]
