"""Blind-Match match schedule (TEST INFRASTRUCTURE ONLY).

The server side of recognition (Sec. 3.3): Input Ciphertext Expansion
(Algorithm 1), HE-C^3 (Algorithm 2), then the compression step, written once
against an evaluator interface (add, mul_plain, mul_cipher, rescale, rotate).
`oracle.ckks.Evaluator` runs it exactly; `CountingEvaluator` only tracks
levels and records (op, level) pairs, which reproduces the cost model F(N_in)
of Sec. 4 (Propositions 1-3 with Table 1).

Readings of passages that are garbled or silent in the paper:

* Algorithm 1's rotation amounts: the printed offset 2^(j + log m - log N_in)
  skips odd sub-windows and at j = log N_in rotates by m (a no-op on data of
  period m), so the replication step here is T_i += Rot(T_i, s * 2^(j-1)),
  j = 1..log2(N_in), always leftwards (the sign alternation is irrelevant for
  period-m data).  After it, slot k of T_i holds q[i*s + (k mod s)].
* The mask of Algorithm 1 selects part i inside every length-m window:
  mask_i[k] = 1 iff floor((k mod m) / s) = i.
* Algorithm 2 rescales every product (Res(Mul(...)) inside the loop); the
  default here accumulates the N_in products and rescales once (same
  message, one rescale instead of N_in).  `rescale_each_part=True` gives the
  printed form.  The loop bound log(m - log N_in) is read as log m - log N_in.
* Compression (the method is only cited; its cost is Proposition 3): each
  group output is masked to the slots k = 0 (mod s) and packed s groups per
  ciphertext, group g going to offset r = g mod s of pack floor(g / s), by a
  radix-2 tree of right rotations (level b: Y_2k + Rot(Y_2k+1, -2^b)), then
  one rescale per pack.  `tree=False` gives the linear form (each group
  rotated right by its offset and added; Proposition 3 charges one Mul, one
  Rot and one Add per group).
"""
import math


def log2i(x):
    v = int(round(math.log2(x)))
    assert 1 << v == x, x
    return v


# ---------------------------------------------------------------------------
# slot layouts (Sec. 3.2 enrollment layout; Sec. 3.3 recognition)
# ---------------------------------------------------------------------------

def tiled_query_slots(q, slots):
    """Query replicated with period m over all slots: z[k] = q[k mod m]."""
    m = len(q)
    return [q[k % m] for k in range(slots)]


def expanded_query_slots(q, s, i, slots):
    """Part i replicated with period s: z[k] = q[i*s + (k mod s)] (client-side expansion)."""
    return [q[i * s + (k % s)] for k in range(slots)]


def gallery_slots(feats, g, i, s, slots):
    """Group g, part i: identity u of the group sits at slots [u*s, u*s+s)
    (z[u*s + t] = g_(g*G+u)[i*s + t], zero past the last identity)."""
    G = slots // s
    R = len(feats)
    z = [0.0] * slots
    for u in range(G):
        idx = g * G + u
        if idx >= R:
            break
        for t in range(s):
            z[u * s + t] = float(feats[idx][i * s + t])
    return z


def gallery_slots_complex(feats, g, i, s, slots):
    """Complex slot packing: group g holds 2G identities; identity u < G of the
    group fills the real parts of slots [u*s, u*s+s), identity G+u the imaginary
    parts of the same slots (the slots of CKKS are complex; the query is real, so
    each part of every product, sum and rotation carries its own identity)."""
    G = slots // s
    R = len(feats)
    z = [0j] * slots
    for u in range(2 * G):
        idx = g * 2 * G + u
        if idx >= R:
            break
        w = u % G
        for t in range(s):
            x = float(feats[idx][i * s + t])
            z[w * s + t] += 1j * x if u >= G else x
    return z


def template_slots(feat, slots):
    """Enrollment ciphertext layout (Sec. 3.2): the vector in the first slots, zeros after."""
    z = [0.0] * slots
    for k, x in enumerate(feat):
        z[k] = float(x)
    return z


def enroll_mask_slots(s, i, slots):
    """Enrollment mask_i (Sec. 3.2): ones at the s slots starting at i*s."""
    return [1.0 if i * s <= k < (i + 1) * s else 0.0 for k in range(slots)]


def alg1_mask_slots(m, s, i, slots):
    """mask_i[k] = 1 iff floor((k mod m)/s) = i."""
    return [1.0 if (k % m) // s == i else 0.0 for k in range(slots)]


def compression_mask_slots(s, slots):
    """M[k] = 1 iff k = 0 (mod s): keeps the slot that holds each identity's score."""
    return [1.0 if k % s == 0 else 0.0 for k in range(slots)]


def n_groups(R, s, slots, complex_pack=False):
    return -(-R // ((2 if complex_pack else 1) * (slots // s)))


def identity_slot(idx, s, slots, packed, complex_pack=False):
    """(output ciphertext, slot, imaginary part?) holding the score of identity idx."""
    G = slots // s
    per = 2 * G if complex_pack else G
    g, w = divmod(idx, per)
    u, im = w % G, w >= G
    if packed:
        p, r = divmod(g, s)
        return p, u * s + r, im
    return g, u * s, im


# ---------------------------------------------------------------------------
# the three stages
# ---------------------------------------------------------------------------

def expand_query(ev, ct, masks, m, s):
    """Algorithm 1: one tiled ciphertext -> N_in ciphertexts, part i replicated."""
    n_in = m // s
    out = []
    for i in range(n_in):
        c = ev.rescale(ev.mul_plain(ct, masks[i]))
        for j in range(1, log2i(n_in) + 1):
            c = ev.add(c, ev.rotate(c, s * (1 << (j - 1))))
        out.append(c)
    return out


def enroll(ev, templates, emasks, s, slots):
    """Sec. 3.2, server side: the encrypted template of identity idx (group g,
    window w) is multiplied by each mask_i (part i), rotated right by (w - i)*s
    slots so that part i lands in window w, and added into the group ciphertext
    C[g][i]; each C[g][i] is rescaled once, after its last identity.  The printed
    shift (Index - i + 1)*m/N_in is read with 0-based indices.  A right rotation
    by t is applied as rotations by the powers of two of t's binary digits,
    lowest first (keys for powers of two only).  Rotating and summing before the
    rescale keeps the key-switching noise of every identity at the product's
    scale Delta*q_L, where it vanishes in the rescale, and adds one rescale's
    rounding per group instead of one per identity.
    Returns C[g][i] for every group that holds an identity."""
    G = slots // s
    n_in = len(emasks)
    groups = -(-len(templates) // G)
    out = [[None] * n_in for _ in range(groups)]
    for idx, ct in enumerate(templates):
        g, w = divmod(idx, G)
        for i in range(n_in):
            x = ev.mul_plain(ct, emasks[i])
            t, b = ((w - i) * s) % slots, 0
            while t:
                if t & 1:
                    x = ev.rotate(x, -(1 << b))
                t >>= 1
                b += 1
            out[g][i] = ev.add(out[g][i], x)
    return [[ev.rescale(c) for c in row] for row in out]


def enroll_rotations(s, slots):
    """Right rotations enrollment uses: every power of two from s below the slot count."""
    return [-(1 << b) for b in range(log2i(s), log2i(slots))]


def expand_query_hoisted(ev, ct, masks, m, s):
    """Algorithm 1's outputs by hoisted rotations (a reordering of the same sum):
    T_i = sum_j Rot(ct (x) mask_i, j*s) over j < N_in, and
    Rot(ct (x) mask_i, j*s) = Rot(ct, j*s) (x) mask_((i-j) mod N_in) because
    shifting by j parts moves part index p to p - j (mod N_in) in every
    length-m window of the tiled query.  The N_in - 1 rotations of the one
    query ciphertext share a basis extension; each T_i is then N_in plaintext
    products summed and rescaled once."""
    n_in = m // s
    rots = [ct] + (ev.rotate_hoisted(ct, [j * s for j in range(1, n_in)]) if n_in > 1 else [])
    out = []
    for i in range(n_in):
        acc = None
        for j in range(n_in):
            acc = ev.add(acc, ev.mul_plain(rots[j], masks[(i - j) % n_in]))
        out.append(ev.rescale(acc))
    return out


def expand_query_fused(ev, ct, m, s):
    """Algorithm 1 with its key switches and rescale fused (same parts as
    expand_query; the bits differ by the roundings saved): the N_in - 1 rotations
    of the query stay in the extended basis Q_L u P before ModDown, the circulant
    mask products run there, and each part is divided once by q_L * P
    (Evaluator.expand_query_fused)."""
    return ev.expand_query_fused(ct, m // s, s, lambda i: alg1_mask_slots(m, s, i, ct_slots(ev)))


def expand_query_ext(ev, ct, m, s):
    """The fused Algorithm 1 up to its division: the N_in sums e_i on Q_L u P
    (Evaluator.expand_query_ext); e_i / (q_L * P) is part i of expand_query_fused."""
    return ev.expand_query_ext(ct, m // s, s, lambda i: alg1_mask_slots(m, s, i, ct_slots(ev)))


def ct_slots(ev):
    return ev.ctx.slots


def bsgs_split(s, double=False):
    """(baby, giant) step counts of the hoisted rotate-and-sum over s (a power of
    two): baby = 2^ceil(log2(s)/2), giant = s / baby.  With one ModDown per
    round output (double=True) a round costs one basis extension, one key-switch
    product per rotation and one ModDown, so up to s = 16 a single round of s - 1
    rotations (baby = s, giant = 1) is cheaper than two."""
    if double and s <= 16:
        return s, 1
    lb = log2i(s)
    b = 1 << ((lb + 1) // 2)
    return b, s // b


def rotsum_hoisted(ev, acc, s, double=False):
    """sum_{r<s} Rot(acc, r) -- the message of Algorithm 2's log2(s)
    rotate-and-add steps -- in two rounds of hoisted rotations: baby steps
    acc + sum_{r<b} Rot(acc, r), then giant steps over multiples of b.
    double=True: each round's rotations summed before one ModDown
    (Evaluator.rotate_sum_hoisted)."""
    b, g = bsgs_split(s, double)
    for step, count in ((1, b), (b, g)):
        if count > 1:
            rs = [step * k for k in range(1, count)]
            if double:
                acc = ev.rotate_sum_hoisted(acc, [(acc, r) for r in rs])
            else:
                for x in ev.rotate_hoisted(acc, rs):
                    acc = ev.add(acc, x)
    return acc


def hec3(ev, cu, cs, s, rescale_each_part=False, encrypted_gallery=False, lazy_relin=True, rotsum="doubling"):
    """Algorithm 2 for one group: sum_i Mul(C_u,i, C_s,i), then log2(s) rotate-and-add steps.

    Slot u*s of the result holds <q, g_u> for every identity u of the group.
    With an encrypted gallery the products are ciphertext x ciphertext; by
    default the tensor products are summed and relinearised once (same
    message, one key switch instead of N_in); lazy_relin=False relinearises
    every product."""
    if encrypted_gallery and lazy_relin and not rescale_each_part:
        acc3 = None
        for i in range(len(cu)):
            acc3 = ev.add3(acc3, ev.tensor(cu[i], cs[i]))
        acc = ev.rescale(ev.relinearize(acc3))
        if rotsum == "none":
            return acc
        if rotsum in ("hoisted", "double"):
            return rotsum_hoisted(ev, acc, s, double=rotsum == "double")
        for t in range(1, log2i(s) + 1):
            acc = ev.add(ev.rotate(acc, 1 << (t - 1)), acc)
        return acc
    mul = ev.mul_cipher if encrypted_gallery else ev.mul_plain
    if rescale_each_part:
        acc = ev.zero_like(cu[0], level=cu[0].level - 1)
        for i in range(len(cu)):
            acc = ev.add(acc, ev.rescale(mul(cu[i], cs[i])))
    else:
        acc = mul(cu[0], cs[0])
        for i in range(1, len(cu)):
            acc = ev.add(acc, mul(cu[i], cs[i]))
        acc = ev.rescale(acc)
    if rotsum == "none":
        return acc
    if rotsum in ("hoisted", "double"):
        return rotsum_hoisted(ev, acc, s, double=rotsum == "double")
    for t in range(1, log2i(s) + 1):
        acc = ev.add(ev.rotate(acc, 1 << (t - 1)), acc)
    return acc


def hec3_deferred(ev, e_parts, cs, s, query_ct, rotsum="doubling"):
    """Algorithm 2 for one group on the undivided parts of the fused Algorithm 1:
    the sum of products on Q_L u P with one division by q_(L-1) * q_L * P
    (Evaluator.hec3_deferred), then the rotate-and-sum as in hec3.  The same
    message as hec3 on expand_query_fused's parts; one division per group in place
    of one per part and the rescale."""
    acc = ev.hec3_deferred(e_parts, cs, query_ct)
    if rotsum == "none":
        return acc
    if rotsum in ("hoisted", "double"):
        return rotsum_hoisted(ev, acc, s, double=rotsum == "double")
    for t in range(1, log2i(s) + 1):
        acc = ev.add(ev.rotate(acc, 1 << (t - 1)), acc)
    return acc


def compress(ev, accs, mask_m, s, tree=True, final_rescale=True, hoisted=False):
    """Compression: mask each group output and pack s groups per ciphertext.
    hoisted=True: the linear form with every group's rotation taken in one
    round (each rotation hoisted: ModUp before the automorphism);
    hoisted="double": the same rotations summed before one ModDown per pack."""
    xs = [ev.mul_plain(a, mask_m) for a in accs]
    packs = []
    for p in range(-(-len(xs) // s)):
        ys = xs[p * s:(p + 1) * s]
        if hoisted == "double":
            y = ev.rotate_sum_hoisted(ys[0], [(ys[r], -r) for r in range(1, len(ys))])
        elif hoisted:
            y = ys[0]
            for r in range(1, len(ys)):
                y = ev.add(y, ev.rotate_hoisted(ys[r], [-r])[0])
        elif tree:
            b = 0
            while len(ys) > 1:
                nxt = []
                for k in range(0, len(ys), 2):
                    if k + 1 < len(ys):
                        nxt.append(ev.add(ys[k], ev.rotate(ys[k + 1], -(1 << b))))
                    else:
                        nxt.append(ys[k])
                ys = nxt
                b += 1
            y = ys[0]
        else:
            y = ev.zero_like(ys[0])
            for r, x in enumerate(ys):
                y = ev.add(y, ev.rotate(x, -r))
        packs.append(ev.rescale(y) if final_rescale else y)
    return packs


def rotsum_compress(ev, accs, mask_m, s):
    """Algorithm 2's rotate-and-sum and the linear compression in one round of
    rotations per pack, with one ModDown per pack (Evaluator.masked_rotate_sums).
    The linear compression puts group o of a pack (o = its offset) at
    Rot(M * acc_o, -o) = Rot(M, -o) * Rot(acc_o, -o), and the rotate-and-sum's last
    round makes acc_o = sum over its rotations k < count of Rot(base_o, step * k), base_o
    the round's input, so Rot(acc_o, -o) = sum_k Rot(base_o, step * k - o): the group's
    terms are the last round's rotations shifted by -o (one of them the identity when o
    is a multiple of step), its plaintext the compression mask rotated by -o.  Rounds
    before the last (the baby steps above s = 16) run as in rotsum_hoisted.  Each pack
    is then rescaled, as the compression's packs are.  The same messages as
    compress(..., hoisted="double") on rotsum_hoisted(double=True)'s outputs; the mask
    multiplies the key-switch sums before ModDown instead of after it, and the groups'
    rotations by -o are no second round."""
    b, g = bsgs_split(s, double=True)
    if g > 1:
        accs = [ev.rotate_sum_hoisted(a, [(a, r) for r in range(1, b)]) for a in accs]
        step, count = b, g
    else:
        step, count = 1, b
    packs = []
    for p in range(-(-len(accs) // s)):
        groups = [(ev.rotate_plaintext(mask_m, -o), [(a, step * k - o) for k in range(count)])
                  for o, a in enumerate(accs[p * s:(p + 1) * s])]
        packs.append(ev.rescale(ev.masked_rotate_sums(groups)))
    return packs


def match(ev, query_cts, gallery_pts, masks, mask_m, m, s, expanded=False,
          rescale_each_part=False, tree=True, encrypted_gallery=False, hoisted=False,
          hoisted_rotsum=False, hoisted_compress=False, double_hoisted=False, fused_compress=False):
    """Full server-side match for one query.

    query_cts: [ct] (tiled, run through Algorithm 1) or the N_in client-expanded cts.
    hoisted: False (the printed doubling order), True (hoisted rotations),
    "fused" (hoisted rotations with their ModDown and the rescale fused) or
    "deferred" (the fused form with its division moved past HE-C^3's products).
    gallery_pts[g][i]: plaintext of group g, part i.
    fused_compress: the rotate-and-sum's last round and the compression in one round
    per pack (rotsum_compress; needs the double-hoisted rotate-and-sum and compression).
    Returns (outputs, packed): the score ciphertexts and whether they are packed."""
    rotsum = ("double" if double_hoisted else "hoisted") if hoisted_rotsum else "doubling"
    if hoisted_compress and double_hoisted:
        hoisted_compress = "double"
    if fused_compress:
        assert rotsum == "double" and hoisted_compress == "double"
        if mask_m is None:
            fused_compress = False

    def tail(accs):
        if fused_compress and accs[0].level >= 1:
            return rotsum_compress(ev, accs, mask_m, s), True
        if fused_compress:
            accs = [rotsum_hoisted(ev, a, s, double=True) for a in accs]
        if accs[0].level >= 1 and mask_m is not None:
            return compress(ev, accs, mask_m, s, tree=tree, hoisted=hoisted_compress), True
        return accs, False
    if fused_compress:
        rotsum = "none"
    if hoisted == "deferred" and not expanded:
        e_parts = expand_query_ext(ev, query_cts[0], m, s)
        accs = [hec3_deferred(ev, e_parts, gallery_pts[g], s, query_cts[0], rotsum=rotsum)
                for g in range(len(gallery_pts))]
        return tail(accs)
    if expanded:
        cu = query_cts
    elif hoisted == "fused":
        cu = expand_query_fused(ev, query_cts[0], m, s)
    elif hoisted:
        cu = expand_query_hoisted(ev, query_cts[0], masks, m, s)
    else:
        cu = expand_query(ev, query_cts[0], masks, m, s)
    accs = [hec3(ev, cu, gallery_pts[g], s, rescale_each_part, encrypted_gallery, rotsum=rotsum)
            for g in range(len(gallery_pts))]
    return tail(accs)


# ---------------------------------------------------------------------------
# op counting (Sec. 4, Propositions 1-3)
# ---------------------------------------------------------------------------

class SymCt:
    def __init__(self, level):
        self.level = level


class CountingEvaluator:
    """Evaluator that only tracks levels and counts (op, input level)."""

    def __init__(self):
        self.ops = []
        self.ctx = None

    def _rec(self, op, level):
        self.ops.append((op, level))

    def add(self, a, b):
        if a is None or b is None:          # the identity of add (as Evaluator.add)
            return b if a is None else a
        self._rec("Add", a.level)
        return SymCt(a.level)

    def mul_plain(self, ct, pt):
        self._rec("MulP", ct.level)
        return SymCt(ct.level)

    def mul_cipher(self, a, b):
        self._rec("MulC", a.level)
        return SymCt(a.level)

    def tensor(self, a, b):
        self._rec("Tensor", a.level)
        return SymCt(a.level)

    def add3(self, x, y):
        if x is not None:
            self._rec("Add", x.level)
        return y

    def relinearize(self, t):
        self._rec("Relin", t.level)
        return SymCt(t.level)

    def rescale(self, ct):
        self._rec("Res", ct.level)
        return SymCt(ct.level - 1)

    def rotate(self, ct, r):
        self._rec("Rot", ct.level)
        return SymCt(ct.level)

    def rotate_hoisted(self, ct, rs):
        self._rec("ModUp", ct.level)
        for r in rs:
            self._rec("RotH", ct.level)
        return [SymCt(ct.level) for _ in rs]

    def expand_query_fused(self, ct, n_in, s, mask_slots):
        L = ct.level
        if n_in > 1:
            self._rec("ModUp", L)
        for _ in range(n_in - 1):
            self._rec("IPH", L)
        self._rec("CircExt", L)
        for _ in range(n_in):
            self._rec("ModDownRes", L)
        return [SymCt(L - 1) for _ in range(n_in)]

    def expand_query_ext(self, ct, n_in, s, mask_slots):
        L = ct.level
        if n_in > 1:
            self._rec("ModUp", L)
        for _ in range(n_in - 1):
            self._rec("IPH", L)
        self._rec("CircExt", L)
        return [SymCt(L) for _ in range(n_in)]

    def hec3_deferred(self, e_parts, pts, ct):
        for _ in e_parts:
            self._rec("MulPExt", ct.level)
        self._rec("ModDownRes2", ct.level)
        return SymCt(ct.level - 2)

    def rotate_sum_hoisted(self, base, terms):
        seen = set()
        rotated = False
        for ct, r in terms:
            if id(ct) not in seen:
                seen.add(id(ct))
                self._rec("ModUp", ct.level)
            self._rec("IPH", ct.level)
            rotated = True
        if rotated:
            self._rec("ModDown", base.level)
        for _ in terms:
            self._rec("Add", base.level)
        return SymCt(base.level)

    def rotate_plaintext(self, pt, r):
        return pt

    def masked_rotate_sums(self, groups):
        lvl = groups[0][1][0][0].level
        seen = set()
        for _, terms in groups:
            for ct, r in terms:
                if r == 0:
                    continue
                if id(ct) not in seen:
                    seen.add(id(ct))
                    self._rec("ModUp", ct.level)
                self._rec("IPH", ct.level)
        self._rec("ModDown", lvl)
        return SymCt(lvl)

    def zero_like(self, ct, level=None):
        return SymCt(ct.level if level is None else level)

    def counts(self):
        out = {}
        for k in self.ops:
            out[k] = out.get(k, 0) + 1
        return out


def paper_literal_ops(n_slots, m, R, n_in, level=3):
    """(op, level) counts of the printed schedule at the paper's setting: encrypted
    gallery (Mul(C)), Res after every product, linear compression without a final
    rescale, ceil(m*R/(n_slots*n_in)) groups served by one expanded query."""
    s = m // n_in
    groups = -(-(m * R // n_slots) // n_in)
    ev = CountingEvaluator()
    masks = [None] * n_in
    cu = expand_query(ev, SymCt(level), masks, m, s)
    accs = [hec3(ev, cu, [SymCt(level - 1)] * n_in, s, rescale_each_part=True,
                 encrypted_gallery=True) for _ in range(groups)]
    compress(ev, accs, None, max(s, groups), tree=False, final_rescale=False)
    return ev.counts()
