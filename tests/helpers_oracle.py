"""Oracle-side construction of match inputs and expected outputs for the parity tests.

Everything here comes from `oracle/` and the seeded generator in
paper_2408_06167_gb300.workload; nothing is read back from the GPU library.
"""
import numpy as np

from oracle import ckks
from oracle import schedule as sch
from paper_2408_06167_gb300 import workload as wl

KEY_SEED = 3
ENC_SEED = 4

_CTX = {}


def octx(name):
    if name not in _CTX:
        _CTX[name] = ckks.Context(name)
    return _CTX[name]


def schedule_rotations(ctx, m, s, hoisted=False, fused_compress=False):
    """Left rotations the tiled/expanded schedule needs (negative = right)."""
    n_in = m // s
    tiled = ctx.L >= 3
    level = ctx.L - 1 if tiled else ctx.L
    rots = []
    if tiled and hoisted:
        rots += [s * j for j in range(1, n_in)]
    elif tiled:
        rots += [s << j for j in range(sch.log2i(n_in))]
    rots += [1 << t for t in range(sch.log2i(s))]
    if level >= 2:
        rots += [-(1 << t) for t in range(sch.log2i(s))]
    if hoisted:
        # both splits of the hoisted rotate-and-sum: one round of 1..s-1, or baby and giant steps
        b, g = sch.bsgs_split(s)
        rots += list(range(1, s)) + [b * k for k in range(1, g)]
        if level >= 2:
            rots += [-r for r in range(1, s)]
    if fused_compress and level >= 2:
        # the last rotate-and-sum round's rotations shifted by every group offset of a pack
        b, g = sch.bsgs_split(s, double=True)
        step, count = (b, g) if g > 1 else (1, b)
        rots += [step * k - o for k in range(count) for o in range(s) if step * k != o]
    return sorted(set(rots), key=rots.index)


class OracleMatch:
    """Keys, gallery plaintexts, query ciphertexts and match outputs from the oracle."""

    def __init__(self, name, m, s, R, n_queries, feats=None, seed=KEY_SEED, complex_pack=False, encrypted=False,
                 hoisted=False, hoisted_tail=False, double_hoisted=False, fused_compress=False):
        self.ctx = ctx = octx(name)
        self.m, self.s, self.R = m, s, R
        self.complex_pack = complex_pack
        self.encrypted = encrypted
        self.hoisted = hoisted
        self.hoisted_tail = hoisted_tail
        self.double_hoisted = double_hoisted
        self.fused_compress = fused_compress
        self.n_in = m // s
        self.tiled = ctx.L >= 3
        self.level = ctx.L - 1 if self.tiled else ctx.L
        self.compress = self.level >= 2
        self.feats = wl.gallery(R, m) if feats is None else feats
        self.queries, self.true_ids = wl.queries(self.feats, n_queries)
        self.sk, self.pk, self.rks = ckks.keygen(ctx, seed, schedule_rotations(ctx, m, s, hoisted or hoisted_tail,
                                                                              fused_compress))
        self.ev = ckks.Evaluator(ctx, self.rks, ckks.keygen_relin(ctx, seed, self.sk) if encrypted else None)
        S, L = ctx.slots, ctx.L
        self.groups = sch.n_groups(R, s, S, complex_pack)
        slots_of = sch.gallery_slots_complex if complex_pack else sch.gallery_slots
        if encrypted:
            # a gallery of ciphertexts at the HE-C^3 level with scale Delta: the packed
            # layout encrypted at the top level (seed 7), top limbs dropped
            def enc(g, i):
                ct = ckks.encrypt(ctx, self.pk, ctx.encode(slots_of(self.feats, g, i, s, S), ctx.scale, L), 7,
                                  g * 256 + i)
                return ckks.Ciphertext(ct.c0[: self.level + 1].copy(), ct.c1[: self.level + 1].copy(), self.level,
                                       ct.scale)
            self.gal = [[enc(g, i) for i in range(self.n_in)] for g in range(self.groups)]
        else:
            self.gal = [[ctx.encode(slots_of(self.feats, g, i, s, S), ctx.q[self.level], self.level)
                         for i in range(self.n_in)] for g in range(self.groups)]
        # scale of the score ciphertexts: one ct x ct product and one rescale with a gallery of ciphertexts
        self.out_scale = ctx.scale ** 2 / ctx.q[self.level] if encrypted else ctx.scale
        self.masks = ([ctx.encode(sch.alg1_mask_slots(m, s, i, S), ctx.q[L], L) for i in range(self.n_in)]
                      if self.tiled else None)
        self.cmask = (ctx.encode(sch.compression_mask_slots(s, S), ctx.q[self.level - 1], self.level - 1)
                      if self.compress else None)

    # arrays in the library's import layouts
    def pts_array(self):
        if self.encrypted:
            return np.stack([np.stack([np.stack([c.c0, c.c1]) for c in row]) for row in self.gal])
        return np.stack([np.stack([p.limbs for p in row]) for row in self.gal])

    def masks_array(self):
        return None if self.masks is None else np.stack([p.limbs for p in self.masks])

    def cmask_array(self):
        return None if self.cmask is None else self.cmask.limbs

    def encrypt(self, qi):
        ctx, S, L = self.ctx, self.ctx.slots, self.ctx.L
        q = self.queries[qi]
        if self.tiled:
            pts = [ctx.encode(sch.tiled_query_slots(q, S), ctx.scale, L)]
        else:
            pts = [ctx.encode(sch.expanded_query_slots(q, self.s, i, S), ctx.scale, L) for i in range(self.n_in)]
        return [ckks.encrypt(ctx, self.pk, pt, ENC_SEED, qi * 256 + k) for k, pt in enumerate(pts)]

    @staticmethod
    def ct_array(cts):
        return np.stack([np.stack([c.c0, c.c1]) for c in cts])

    def match(self, cts):
        outs, packed = sch.match(self.ev, cts, self.gal, self.masks, self.cmask, self.m, self.s,
                                 expanded=not self.tiled, encrypted_gallery=self.encrypted,
                                 hoisted=self.hoisted, hoisted_rotsum=self.hoisted_tail,
                                 hoisted_compress=self.hoisted_tail, double_hoisted=self.double_hoisted,
                                 fused_compress=self.fused_compress)
        return self.ct_array(outs), packed

    def scores(self, outs_array, packed):
        ctx, S = self.ctx, self.ctx.slots
        dec = []
        for o in outs_array:
            ct = ckks.Ciphertext(o[0], o[1], 0, self.out_scale)
            dec.append(ckks.decrypt_decode(ctx, ct, self.sk))
        return np.array([dec[o][slot].imag if im else dec[o][slot].real
                         for o, slot, im in (sch.identity_slot(i, self.s, S, packed, self.complex_pack)
                                             for i in range(self.R))])
