"""Hand-built models shared by the oracle pins and the GPU parity tests."""
import numpy as np


def fp8_exact_model():
    """A page model on which every FP8 quantisation is exact, with a layer-1 unit at the 448 edge.

    Features at full resolution read at texel centres are exactly 0 or 1
    (six-value BC4 mode, literal indices 6 and 7); the temporal line holds 0
    or 1 and is read at keyframes; weights, biases and every hidden value have
    at most four significant bits and stay inside E4M3's normal range at the
    chosen scales.  Layer 1 sees a spatial term (one weight per unit), a
    temporal term (0.5 on one temporal channel, every unit but 0) and b1 in
    {0, 0.5}, so z1 is a multiple of 0.5 up to 2.5, or 3.5 for unit 0 (which
    lands on E4M3's largest value); z2 is a multiple of 1/8 up to 1.875.
    """
    rng = np.random.default_rng(11)
    cs, ct, T, H, fw = 16, 8, 8, 32, 32
    bc4 = np.zeros((fw // 4, fw // 4, cs, 8), np.uint8)
    bc4[..., 0], bc4[..., 1] = 10, 200                 # r0 <= r1: six-value mode
    idx = rng.choice([6, 7], size=(fw // 4, fw // 4, cs, 16))
    bits = np.zeros(idx.shape[:-1], np.uint64)
    for p in range(16):
        bits |= idx[..., p].astype(np.uint64) << np.uint64(3 * p)
    for k in range(6):
        bc4[..., 2 + k] = ((bits >> np.uint64(8 * k)) & np.uint64(0xFF)).astype(np.uint8)
    temporal = rng.choice([0.0, 1.0], size=(T, ct)).astype(np.float32)
    w1 = np.zeros((cs + ct, H), np.float32)
    for o in range(H):
        w1[o % cs, o] = rng.choice([0.5, 1.0, 1.5, -1.0])
        if o > 0:
            w1[cs + o % ct, o] = 0.5
    w1[0, 0] = 3.5
    b1 = rng.choice([0.0, 0.5], size=H).astype(np.float32)
    b1[0] = 0.0
    w2 = np.zeros((H, H), np.float32)
    for o in range(H):
        w2[o, o] = rng.choice([0.25, 0.5])
    b2 = rng.choice([0.0, 0.125], size=H).astype(np.float32)
    w3 = rng.choice([-0.5, 0.5, 1.0], size=(H, 3)).astype(np.float32)
    b3 = np.array([0.5, -0.25, 0.125], np.float32)
    return dict(lm_w=fw, lm_h=fw, feat_w=fw, feat_h=fw, cs=cs, bc4=bc4, t_count=T, ct=ct, temporal=temporal,
                hidden=H, w1=w1, b1=b1, w2=w2, b2=b2, w3=w3, b3=b3, address_mode=0)
