"""A CPU model of the merge kernel's round protocol (test infrastructure).

The CUDA kernel certifies several consecutive merges of the Section 4
iteration per pair of grid barriers.  This module replays the same protocol
on the host, one round at a time, with the kernel's data structures:

* per row a cache of the K smallest keys (value, column) over live columns to
  its right, and a bound B (every live cell outside the cache is above B);
* per CTA (rows dealt in blocks of 32, round-robin) the `pub` smallest
  entries of its rows' caches, each row's cached keys followed by a stop mark
  at B, the last published entry a hard stop;
* the walk over the union of the published lists, the chain of disjoint
  pairs, the new cells computed before anything is written, the certified
  prefix, the bookkeeping (survivor caches from the smallest new cell to the
  right and the cells between chain members), and the refills (requested when
  a cache holds `refill_at` keys or fewer, scanned one round later, installed
  the round after with the merges in between replayed) or, for one CTA, the
  immediate refresh.

It shares no code with the oracle or the library.  Tests compare its output
with the oracle bit for bit, and a planted mistake (accepting the whole chain
without certification) must be caught.  Arithmetic: IEEE binary32 with every
operation rounded, terms in printed order (Section 4 step 3, Table 1).
"""
from __future__ import annotations

import numpy as np

K = 4            # cached keys per row
MAX_REQ = 256    # refill rows served per round
REQ_PER_CTA = 8
NOKEY = (1 << 64) - 1
f32 = np.float32


def _bits(v) -> int:
    return int(np.float32(v).view(np.uint32))


def _key(v, c) -> int:
    return (_bits(v) << 32) | int(c)


def lw_cell(linkage, dki, dkj, dij, ni, nj, nk):
    dki, dkj, dij = f32(dki), f32(dkj), f32(dij)
    ai = aj = f32(0.5)
    be = ga = f32(0.0)
    if linkage == 0:
        ga = f32(-0.5)
    elif linkage == 1:
        ga = f32(0.5)
    elif linkage in (2, 5):
        sm = f32(ni + nj)
        ai, aj = f32(ni) / sm, f32(nj) / sm
        if linkage == 5:
            be = -(f32(ni * nj) / f32((ni + nj) * (ni + nj)))
    elif linkage == 3:
        t = f32(ni + nj + nk)
        ai, aj, be = f32(ni + nk) / t, f32(nj + nk) / t, -(f32(nk) / t)
    # 4, weighted average: 1/2, 1/2, 0, 0
    s = f32(ai * dki)
    s = f32(s + f32(aj * dkj))
    s = f32(s + f32(be * dij))
    return f32(s + f32(ga * abs(f32(dki - dkj))))


class RoundModel:
    def __init__(self, packed, n, linkage, G=1, chain=16, pub=4, certify=True, refill_at=0, scan=False):
        self.n, self.link, self.G = n, linkage, G
        # scan: certify as the kernel does (per merge a, a suffix minimum over
        # the pairs c >= p and an exclusive prefix minimum over a < c < p),
        # instead of the direct loops over (p, a, c)
        self.scan = scan
        self.decisions = []
        self.refill_at = refill_at
        self.chain = chain
        self.pub = pub
        self.certify = certify
        M = np.zeros((n, n), dtype=np.float32)
        iu = np.triu_indices(n, 1)
        M[iu] = packed
        M[(iu[1], iu[0])] = packed
        self.M = M
        self.live = np.ones(n, dtype=bool)
        self.size = np.ones(n, dtype=np.int64)
        self.cache = {}
        self.bound = {}
        self.pend = {}      # row -> round of its refill request
        for r in range(n):
            self._fill(r)

    # ---- row caches
    def _row_keys(self, r):
        return sorted(_key(self.M[r, c], c) for c in range(r + 1, self.n) if self.live[c])

    def _fill(self, r):
        ks = self._row_keys(r)
        self.cache[r] = ks[:K]
        self.bound[r] = ks[K - 1] if len(ks) >= K else NOKEY
        if len(self.cache[r]) == K:
            self.bound[r] = self.cache[r][K - 1]

    def _owner(self, r):
        return (r // 32) % self.G

    # ---- published entries of one CTA: (order key, column word)
    def _publish(self, g):
        ents = []
        for r in range(self.n):
            if self._owner(r) != g or not self.live[r]:
                continue
            c = len(self.cache[r])
            for q, k in enumerate(self.cache[r]):
                ents.append((((k >> 32) << 32) | (r << 3) | q, ("col", k & 0xFFFFFFFF)))
            if self.bound[r] != NOKEY:
                ents.append((((self.bound[r] >> 32) << 32) | (r << 3) | c, ("rowstop", None)))
        ents.sort(key=lambda e: e[0])
        top = ents[:self.pub]
        if len(top) == self.pub:
            top[-1] = (top[-1][0], top[-1][1] + ("hard",))
        return top

    def _walk(self, recs):
        ents = sorted((e for rec in recs for e in rec), key=lambda e: e[0])
        chain, touched = [], set()
        for okey, word in ents:
            row = (okey & 0xFFFFFFFF) >> 3
            stop = len(word) > 2
            if row not in touched:
                if word[0] == "rowstop":
                    stop = True
                elif word[1] not in touched:
                    c = word[1]
                    chain.append((row, c, f32(np.uint32(okey >> 32).view(np.float32))))
                    touched |= {row, c}
                    if len(chain) == self.chain:
                        stop = True
            if stop:
                break
        return chain

    def run(self):
        n, M = self.n, self.M
        merges, heights = [], []
        t, rnd = 0, 0
        served = {}          # round -> {row: scanned keys}
        requests = {}        # round -> rows that asked in that round
        prev = []            # merges of the previous round
        while t < n - 1:
            if rnd > 2 * n + 64:
                raise RuntimeError("no progress")
            recs = [self._publish(g) for g in range(self.G)]
            # refills asked for in round rnd - 1 are scanned now (state after it)
            exec_rows = requests.get(rnd - 1, [])[:MAX_REQ]
            served[rnd] = {r: [k for k in self._row_keys(r)][:K] for r in exec_rows}
            # ... and the ones scanned in round rnd - 1 are installed, with the
            # merges of round rnd - 1 replayed
            for r, keys in served.get(rnd - 1, {}).items():
                if self.pend.get(r) != rnd - 2 or not self.live[r]:
                    continue
                c = len(keys)
                B = keys[K - 1] if c == K else NOKEY
                ks = [k for k in keys if all((k & 0xFFFFFFFF) not in (a, b) for a, b in prev)]
                c = len(ks)
                for a, _ in prev:
                    if a > r:
                        x = _key(M[r, a], a)
                        if x <= B:
                            ks = sorted(ks + [x])
                            if c == K:
                                ks = ks[:K]
                                B = ks[K - 1]
                            else:
                                c += 1
                self.cache[r], self.bound[r] = ks, B
                del self.pend[r]
            chain = self._walk(recs)
            s = len(chain)
            members = {x for a, b, _ in chain for x in (a, b)}
            szi = [int(self.size[a]) for a, _, _ in chain]
            szj = [int(self.size[b]) for _, b, _ in chain]
            # pass 1: new cells outside the chain (nothing written yet)
            amin, hmin = [NOKEY] * s, [NOKEY] * s
            for k in range(n):
                if not self.live[k] or k in members:
                    continue
                for a, (ia, ja, h) in enumerate(chain):
                    v = lw_cell(self.link, M[k, ia], M[k, ja], h, szi[a], szj[a], int(self.size[k]))
                    kk = _key(v, k)
                    amin[a] = min(amin[a], kk)
                    if k > ia:
                        hmin[a] = min(hmin[a], kk)
            X, Y, C = {}, {}, {}
            for a, (ia, ja, h) in enumerate(chain):
                for c, (ib, jb, _) in enumerate(chain):
                    if a != c:
                        X[a, c] = lw_cell(self.link, M[ib, ia], M[ib, ja], h, szi[a], szj[a], szi[c])
                        Y[a, c] = lw_cell(self.link, M[jb, ia], M[jb, ja], h, szi[a], szj[a], szj[c])
            for a in range(s):
                for c in range(a + 1, s):
                    C[a, c] = lw_cell(self.link, X[a, c], Y[a, c], chain[c][2], szi[c], szj[c], szi[a] + szj[a])
            # certification: P_{p+1} below every cell merges 0..p rewrote
            L = s
            if self.certify and self.scan:
                def cell(vb, x, y):
                    return (vb, min(x, y), max(x, y))
                none = (1 << 40, 0, 0)
                R = {}
                for a in range(s - 1):
                    ia = chain[a][0]
                    suf = [none] * (s + 1)
                    for c in range(s - 1, a, -1):
                        suf[c] = min(suf[c + 1], cell(_bits(X[a, c]), ia, chain[c][0]),
                                     cell(_bits(Y[a, c]), ia, chain[c][1]))
                    g = cell(amin[a] >> 32, ia, amin[a] & 0xFFFFFFFF) if amin[a] != NOKEY else none
                    pre = none
                    for c in range(a + 1, s):
                        R[a, c] = min(g, suf[c], pre)
                        pre = min(pre, cell(_bits(C[a, c]), ia, chain[c][0]))
                for pp in range(1, s):
                    P = (_bits(chain[pp][2]), chain[pp][0], chain[pp][1])
                    if not P < min(R[a, pp] for a in range(pp)):
                        L = pp
                        break
            elif self.certify:
                def cell(vb, x, y):
                    return (vb, min(x, y), max(x, y))
                for pp in range(1, s):
                    P = (_bits(chain[pp][2]), chain[pp][0], chain[pp][1])
                    low = (1 << 40, 0, 0)
                    for a in range(pp):
                        ia = chain[a][0]
                        if amin[a] != NOKEY:
                            low = min(low, cell(amin[a] >> 32, ia, amin[a] & 0xFFFFFFFF))
                        for c in range(pp, s):
                            low = min(low, cell(_bits(X[a, c]), ia, chain[c][0]),
                                      cell(_bits(Y[a, c]), ia, chain[c][1]))
                        for c in range(a + 1, pp):
                            low = min(low, cell(_bits(C[a, c]), ia, chain[c][0]))
                    if not P < low:
                        L = pp
                        break
            self.decisions.append((s, L))
            # bookkeeping of the L merges
            for a in range(L):
                merges.append((chain[a][0], chain[a][1]))
                heights.append(chain[a][2])
            for a in range(L):
                for c in range(a + 1, L):
                    M[chain[a][0], chain[c][0]] = M[chain[c][0], chain[a][0]] = C[a, c]
            merged = {x for a, b, _ in chain[:L] for x in (a, b)}
            asked = []
            for a in range(L):
                ia, ja, _ = chain[a]
                self.live[ja] = False
                self.cache[ja], self.bound[ja] = [], NOKEY
                self.pend.pop(ja, None)
                self.pend.pop(ia, None)
            refresh = []
            for a in range(L):
                ia = chain[a][0]
                if self.G == 1:
                    refresh.append(ia)
                    continue
                m = hmin[a]
                cands = []
                for c in range(s):
                    if c == a:
                        continue
                    ib, jb, _ = chain[c]
                    if c < L:
                        if ib > ia:
                            cands.append(_key(C[min(a, c), max(a, c)], ib))
                    else:
                        if ib > ia:
                            cands.append(_key(X[a, c], ib))
                        if jb > ia:
                            cands.append(_key(Y[a, c], jb))
                if m != NOKEY:
                    ks = sorted([x for x in cands if x < m] + [m])[:K]
                    B = ks[-1]
                else:
                    ks = sorted(cands)[:K]
                    B = ks[K - 1] if len(cands) > K else NOKEY
                self.cache[ia], self.bound[ia] = ks, B
                if len(ks) <= self.refill_at and B != NOKEY:
                    asked.append(ia)
            # pass 2: write the new cells, keep the caches
            for k in range(n):
                if not self.live[k] or k in merged:
                    continue
                ks, B = list(self.cache[k]), self.bound[k]
                for a in range(L):
                    ia, ja, h = chain[a]
                    v = lw_cell(self.link, M[k, ia], M[k, ja], h, szi[a], szj[a], int(self.size[k]))
                    M[k, ia] = M[ia, k] = v
                    if k < ja:
                        ks = [x for x in ks if (x & 0xFFFFFFFF) != ja and not (k < ia and (x & 0xFFFFFFFF) == ia)]
                        c = len(ks)
                        if k < ia:
                            x = _key(v, ia)
                            if x <= B:
                                ks = sorted(ks + [x])
                                if c == K:
                                    ks = ks[:K]
                                    B = ks[K - 1]
                                else:
                                    c += 1
                self.cache[k], self.bound[k] = ks, B
                if self.G == 1:
                    if len(ks) <= self.refill_at and B != NOKEY:
                        refresh.append(k)
                elif len(ks) <= self.refill_at and B != NOKEY and k not in self.pend:
                    asked.append(k)
            for a in range(L):
                self.size[chain[a][0]] = szi[a] + szj[a]
            for r in refresh:       # one CTA sees every write: rescan now
                self._fill(r)
            # requests, at most REQ_PER_CTA per CTA, in CTA order
            per = {}
            kept = []
            for r in sorted(asked, key=lambda r: self._owner(r)):
                g = self._owner(r)
                if per.get(g, 0) < REQ_PER_CTA:
                    per[g] = per.get(g, 0) + 1
                    kept.append(r)
                    self.pend[r] = rnd
            requests[rnd] = kept
            prev = [(chain[a][0], chain[a][1]) for a in range(L)]
            t += L
            rnd += 1
        return np.array(merges, dtype=np.int32).reshape(-1, 2), np.array(heights, dtype=np.float32), rnd
