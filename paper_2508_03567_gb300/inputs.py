"""Seeded synthetic workloads for non-binary LDPC min-max decoding.

This module makes decoder *inputs* and nothing else: sparse parity-check
matrices H over GF(2^p), transmitted codewords, and the quantized symbol
reliabilities gamma [frames, N, q] (uint8) that a decoder consumes.  It holds
none of the decoder's arithmetic (no check-node, variable-node, decision or
syndrome step).  Both the CPU oracle and the CUDA decoder read what it makes;
neither side's code is used here.

The paper's own codes (CCSDS-derived (16,8)/(32,16)/(64,32) codes, Sec. 5)
are not available, so seeded random regular codes stand in for them:

* H: socket (stub) permutation of N*d_v variable sockets onto M*d_c check
  sockets, then local repair by random socket swaps until no check meets the
  same variable twice and no two variables share two checks (girth > 4);
  coefficients uniform in GF(q)\\{0}.  The code definition follows Sec. 2.1
  (M x N sparse H, regular when row and column weights are constant).
* Codewords: random information symbols on the non-pivot columns of the
  reduced row-echelon form of H over GF(q); pivot symbols solved.  The field
  multiply used for this (carry-less product reduced by the primitive
  polynomial) is private to codeword construction.
* Channel: BPSK (bit b -> 1 - 2b, bit i of a symbol is (a >> i) & 1) over
  AWGN with sigma^2 = 1 / (2 R 10^(EbN0/10)), R = K/N; bit LLR 2y/sigma^2;
  symbol reliability relative to the hard decision (Sec. 2.2 and the
  initialization of Alg. 2): gamma(a) = sum of |LLR_i| over the bits where a
  disagrees with the hard decision, then x4, round half to even, cap 63.

All floating-point steps are elementwise IEEE operations in a fixed order, so
the same seed gives bit-identical gamma on CPU and GPU.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
import torch

# Primitive polynomials (bit i = coefficient of x^i), one per field order.
PRIMITIVE_POLY = {
    2: 0x3,      # x + 1
    4: 0x7,      # x^2 + x + 1
    8: 0xB,      # x^3 + x + 1
    16: 0x13,    # x^4 + x + 1
    32: 0x25,    # x^5 + x^2 + 1
    64: 0x43,    # x^6 + x + 1
    128: 0x83,   # x^7 + x + 1
    256: 0x11D,  # x^8 + x^4 + x^3 + x^2 + 1
}

NOISE_BLOCK = 1024  # frames per independently seeded RNG block


# ----------------------------------------------------------------------------
# Field multiply for codeword construction only.
# ----------------------------------------------------------------------------
def _clmul_reduce(a: int, b: int, q: int, poly: int) -> int:
    """Carry-less product of a and b reduced modulo the primitive polynomial."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a & q:
            a ^= poly
    return r


def _mul_table(q: int, poly: int) -> np.ndarray:
    t = np.zeros((q, q), dtype=np.int64)
    for a in range(q):
        for b in range(a, q):
            t[a, b] = t[b, a] = _clmul_reduce(a, b, q, poly)
    return t


# ----------------------------------------------------------------------------
# Codes
# ----------------------------------------------------------------------------
@dataclass
class Code:
    q: int
    poly: int
    n: int
    m: int
    row_ptr: np.ndarray   # int32 [m+1]
    col_idx: np.ndarray   # int32 [nnz]
    coef: np.ndarray      # uint8 [nnz], 1..q-1
    name: str = ""
    rank: int = -1
    pivots: np.ndarray = field(default=None, repr=False)   # pivot columns of RREF
    free: np.ndarray = field(default=None, repr=False)     # non-pivot columns
    _gbin: torch.Tensor = field(default=None, repr=False)  # info bits -> pivot bits

    @property
    def p(self) -> int:
        return int(self.q).bit_length() - 1

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def k(self) -> int:
        return self.n - self.rank

    def dense(self) -> np.ndarray:
        h = np.zeros((self.m, self.n), dtype=np.int64)
        for r in range(self.m):
            for e in range(self.row_ptr[r], self.row_ptr[r + 1]):
                h[r, self.col_idx[e]] = self.coef[e]
        return h


def code_from_dense(h: np.ndarray, q: int, poly: int, name: str = "") -> Code:
    """CSR code from a dense coefficient matrix (rows in order, columns ascending)."""
    h = np.asarray(h)
    m, n = h.shape
    rp = [0]
    ci, cf = [], []
    for r in range(m):
        for c in range(n):
            if h[r, c]:
                ci.append(c)
                cf.append(int(h[r, c]))
        rp.append(len(ci))
    code = Code(q=q, poly=poly, n=n, m=m, row_ptr=np.array(rp, np.int32),
                col_idx=np.array(ci, np.int32), coef=np.array(cf, np.uint8), name=name)
    _finish(code)
    return code


def _bad_edges(edge_vn: np.ndarray, m: int, dc: int) -> list[int]:
    """Edges whose variable repeats within a check or closes a 4-cycle."""
    bad = set()
    rows = edge_vn.reshape(m, dc)
    checks_of = {}
    for c in range(m):
        seen = {}
        for j in range(dc):
            v = int(rows[c, j])
            e = c * dc + j
            if v in seen:
                bad.add(e)
            else:
                seen[v] = e
                checks_of.setdefault(v, []).append((c, e))
    pair_owner = {}
    for v in sorted(checks_of):
        lst = checks_of[v]
        for a in range(len(lst)):
            for b in range(a + 1, len(lst)):
                c1, e1 = lst[a]
                c2, e2 = lst[b]
                key = (min(c1, c2), max(c1, c2))
                if key in pair_owner:
                    bad.add(e2)
                else:
                    pair_owner[key] = v
    return sorted(bad)


def make_regular_code(q: int, n: int, dv: int, dc: int, seed: int, poly: int | None = None,
                      name: str = "", max_rounds: int = 20000, encoder: bool = True) -> Code:
    """Seeded regular (dv, dc) code over GF(q) with girth > 4 (see module doc).

    encoder=False skips the row reduction (no codewords can be drawn; rank stays -1):
    for large codes decoded from random reliabilities."""
    poly = PRIMITIVE_POLY[q] if poly is None else poly
    e_total = n * dv
    if e_total % dc:
        raise ValueError("n*dv must be a multiple of dc")
    m = e_total // dc
    rng = np.random.Generator(np.random.PCG64(seed))
    edge_vn = np.repeat(np.arange(n, dtype=np.int64), dv)[rng.permutation(e_total)]
    for _ in range(max_rounds):
        bad = _bad_edges(edge_vn, m, dc)
        if not bad:
            break
        for e in bad:
            f = int(rng.integers(e_total))
            edge_vn[e], edge_vn[f] = edge_vn[f], edge_vn[e]
    else:
        raise RuntimeError(f"socket repair did not converge for seed {seed}")
    rows = np.sort(edge_vn.reshape(m, dc), axis=1)
    coef = rng.integers(1, q, size=e_total).astype(np.uint8)
    code = Code(q=q, poly=poly, n=n, m=m,
                row_ptr=(np.arange(m + 1, dtype=np.int32) * dc),
                col_idx=rows.reshape(-1).astype(np.int32), coef=coef, name=name)
    if encoder:
        _finish(code)
    return code


def _finish(code: Code) -> None:
    """Row-reduce H over GF(q) (leftmost pivots) and build the bit-level encoder."""
    q, p = code.q, code.p
    mul = _mul_table(q, code.poly)
    inv = np.zeros(q, dtype=np.int64)
    for a in range(1, q):
        inv[a] = int(np.nonzero(mul[a] == 1)[0][0])
    h = code.dense()
    r = 0
    pivots = []
    for c in range(code.n):
        if r == code.m:
            break
        nz = np.nonzero(h[r:, c])[0]
        if nz.size == 0:
            continue
        piv = r + int(nz[0])
        if piv != r:
            h[[r, piv]] = h[[piv, r]]
        h[r] = mul[inv[h[r, c]], h[r]]
        for rr in range(code.m):
            if rr != r and h[rr, c]:
                h[rr] ^= mul[h[rr, c], h[r]]
        pivots.append(c)
        r += 1
    code.rank = r
    code.pivots = np.array(pivots, dtype=np.int64)
    code.free = np.array([c for c in range(code.n) if c not in set(pivots)], dtype=np.int64)
    # c[pivot_r] = sum over free f of R[r, f] * c[f]  (characteristic 2)
    k = code.free.size
    coefs = h[:r][:, code.free]                          # [rank, K]
    mulbits = mul[:, [1 << i for i in range(p)]]        # [q, p]: g * x^i
    vals = mulbits[coefs]                                # [rank, K, p_in]
    bits = (vals[..., None] >> np.arange(p)) & 1         # [rank, K, p_in, p_out]
    g = bits.transpose(1, 2, 0, 3).reshape(k * p, r * p)
    code._gbin = torch.from_numpy(g.astype(np.float32))


def _bits(sym: torch.Tensor, p: int) -> torch.Tensor:
    sh = torch.arange(p, device=sym.device)
    return (sym.to(torch.int64)[..., None] >> sh) & 1


def encode(code: Code, info: torch.Tensor) -> torch.Tensor:
    """Codewords [F, N] (int64) for information symbols info [F, K] on the free columns."""
    dev = info.device
    p, f = code.p, info.shape[0]
    c = torch.zeros((f, code.n), dtype=torch.int64, device=dev)
    c[:, torch.from_numpy(code.free).to(dev)] = info.to(torch.int64)
    if code.rank:
        ib = _bits(info, p).reshape(f, -1).to(torch.float32)
        # 0/1 products summed in fp32: exact for sums < 2^24, on any device.
        pb = torch.remainder(ib @ code._gbin.to(dev), 2.0).to(torch.int64)
        pb = pb.reshape(f, code.rank, p)
        ps = (pb << torch.arange(p, device=dev)).sum(-1)
        c[:, torch.from_numpy(code.pivots).to(dev)] = ps
    return c


# ----------------------------------------------------------------------------
# Channel and quantizer
# ----------------------------------------------------------------------------
def sigma2_for(code: Code, ebn0_db: float) -> float:
    rate = code.k / code.n
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def _block_rng(seed: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, block])))


def _blocks(frame0: int, frames: int):
    b0 = frame0 // NOISE_BLOCK
    b1 = (frame0 + frames + NOISE_BLOCK - 1) // NOISE_BLOCK
    for b in range(b0, b1):
        lo = max(frame0, b * NOISE_BLOCK)
        hi = min(frame0 + frames, (b + 1) * NOISE_BLOCK)
        yield b, lo - b * NOISE_BLOCK, hi - b * NOISE_BLOCK


def info_symbols(code: Code, seed: int, frame0: int, frames: int) -> torch.Tensor:
    out = []
    for b, lo, hi in _blocks(frame0, frames):
        rng = _block_rng(seed, b)
        blk = rng.integers(0, code.q, size=(NOISE_BLOCK, code.k))
        out.append(blk[lo:hi])
    return torch.from_numpy(np.concatenate(out, 0) if out else np.zeros((0, code.k), np.int64))


def awgn(code: Code, seed: int, frame0: int, frames: int) -> torch.Tensor:
    """Standard normal samples [frames, N, p] (float64), block-seeded."""
    out = []
    for b, lo, hi in _blocks(frame0, frames):
        rng = _block_rng(seed, b)
        blk = rng.standard_normal(size=(NOISE_BLOCK, code.n, code.p))
        out.append(blk[lo:hi])
    return torch.from_numpy(np.concatenate(out, 0) if out else np.zeros((0, code.n, code.p)))


def _symbol_costs(code: Code, codewords: torch.Tensor, noise: torch.Tensor, ebn0_db) -> torch.Tensor:
    """g [F, N, q] float64: sum of |LLR_i| over the bits i where symbol x differs
    from the bitwise hard decision (BPSK bit 0 -> +1, AWGN, LLR = 2y / sigma^2).

    ebn0_db is one value for every frame or a float64 tensor [F] of per-frame values."""
    dev = codewords.device
    q, p = code.q, code.p
    if isinstance(ebn0_db, torch.Tensor):
        rate = code.k / code.n
        s2 = (1.0 / (2.0 * rate * torch.pow(10.0, ebn0_db.to(torch.float64) / 10.0))).to(dev)[:, None, None]
        sigma = torch.sqrt(s2)
    else:
        s2 = sigma2_for(code, ebn0_db)
        sigma = math.sqrt(s2)
    b = _bits(codewords, p).to(torch.float64)
    s = 1.0 - 2.0 * b
    y = s + sigma * noise.to(dev)
    llr = (2.0 * y) / s2
    mag = llr.abs()
    hard = ((y < 0).to(torch.int64) << torch.arange(p, device=dev)).sum(-1)  # [F, N]
    # t[u] = sum of mag_i over the set bits i of u, added in increasing i.
    t = torch.zeros(codewords.shape + (q,), dtype=torch.float64, device=dev)
    for i in range(p):
        w = 1 << i
        t[..., w:2 * w] = t[..., 0:w] + mag[..., i:i + 1]
    idx = torch.arange(q, device=dev) ^ hard[..., None]
    return torch.gather(t, -1, idx)


def quantized_reliabilities(code: Code, codewords: torch.Tensor, noise: torch.Tensor,
                            ebn0_db) -> torch.Tensor:
    """gamma [F, N, q] uint8 from codewords [F, N] and unit noise [F, N, p]:
    min(63, round(4 g)) of the symbol costs g (0 for the most likely symbol)."""
    g = _symbol_costs(code, codewords, noise, ebn0_db)
    return torch.clamp(torch.round(4.0 * g), max=63.0).to(torch.uint8)


def channel_probabilities(code: Code, codewords: torch.Tensor, noise: torch.Tensor,
                          ebn0_db) -> torch.Tensor:
    """p [F, N, q] float32: the symbol probabilities p(c_n = x | y_n), the product
    of the independent bit probabilities, normalized to sum 1 (computed in
    float64 as exp(-g) / sum exp(-g), then rounded to float32)."""
    g = _symbol_costs(code, codewords, noise, ebn0_db)
    w = torch.exp(-g)
    return (w / w.sum(-1, keepdim=True)).to(torch.float32)


def frame_ebn0(seed: int, frame0: int, frames: int, lo: float, hi: float) -> torch.Tensor:
    """Per-frame Eb/N0 in dB, uniform in [lo, hi), block-seeded like the noise."""
    out = []
    for b, a, z in _blocks(frame0, frames):
        rng = _block_rng(seed, b)
        out.append(lo + (hi - lo) * rng.random(NOISE_BLOCK)[a:z])
    return torch.from_numpy(np.concatenate(out) if out else np.zeros(0))


@dataclass
class Batch:
    gamma: torch.Tensor       # [F, N, q] uint8
    codewords: torch.Tensor   # [F, N] int64
    prob: torch.Tensor | None = None   # [F, N, q] float32 channel probabilities (make_batch(prob=True))


def make_batch(code: Code, ebn0_db, seed: int, frames: int, frame0: int = 0,
               device: str | torch.device = "cpu", noiseless: bool = False,
               chunk: int = 4096, prob: bool = False) -> Batch:
    """Frames [frame0, frame0+frames) of one (code, Eb/N0, seed) stream.

    ebn0_db: one value, or a (lo, hi) pair for per-frame Eb/N0 uniform in [lo, hi).
    prob: also return the float32 channel probabilities of the same frames."""
    gam, cws, prs = [], [], []
    for lo in range(0, frames, chunk):
        nf = min(chunk, frames - lo)
        info = info_symbols(code, seed, frame0 + lo, nf).to(device)
        cw = encode(code, info)
        if noiseless:
            nz = torch.zeros(cw.shape + (code.p,), dtype=torch.float64)
        else:
            nz = awgn(code, seed + 1, frame0 + lo, nf)
        eb = frame_ebn0(seed + 2, frame0 + lo, nf, *ebn0_db) if isinstance(ebn0_db, tuple) else ebn0_db
        gam.append(quantized_reliabilities(code, cw, nz, eb))
        cws.append(cw)
        if prob:
            prs.append(channel_probabilities(code, cw, nz, eb))
    if not gam:
        return Batch(torch.zeros((0, code.n, code.q), dtype=torch.uint8, device=device),
                     torch.zeros((0, code.n), dtype=torch.int64, device=device),
                     torch.zeros((0, code.n, code.q), dtype=torch.float32, device=device) if prob else None)
    return Batch(torch.cat(gam, 0), torch.cat(cws, 0), torch.cat(prs, 0) if prob else None)


# ----------------------------------------------------------------------------
# Workloads (the decode workloads the benchmarks and parity tests run)
# ----------------------------------------------------------------------------
WORKLOADS = {
    # GF(4) rate-1/2 (2,4) N=48, 1000 frames at 3 dB, 10 fixed iterations.
    "gf4_n48_dv2_dc4": dict(q=4, n=48, dv=2, dc=4, code_seed=1101, data_seed=1201,
                            frames=1000, ebn0=(3.0,), max_iters=10, early_stop=0),
    # GF(64) rate-1/2 (2,4) N=576, 65536 frames at each of 1.5/2.0/2.5 dB, <=20 its.
    "gf64_n576_dv2_dc4": dict(q=64, n=576, dv=2, dc=4, code_seed=2101, data_seed=2201,
                              frames=65536, ebn0=(1.5, 2.0, 2.5), max_iters=20, early_stop=1),
    # GF(256) rate-2/3 (2,6) N=384, 16384 frames at 2.5 dB, <=20 its.
    "gf256_n384_dv2_dc6": dict(q=256, n=384, dv=2, dc=6, code_seed=3101, data_seed=3201,
                               frames=16384, ebn0=(2.5,), max_iters=20, early_stop=1),
    # Mixed-code set: GF(16) (2,4) N=1024; GF(64) (2,4) N=576; GF(32) (3,6) N=600;
    # GF(256) (2,8) N=128; up to 30 iterations.
    "gf16_n1024_dv2_dc4": dict(q=16, n=1024, dv=2, dc=4, code_seed=4101, data_seed=4201,
                               frames=4096, ebn0=(1.5, 3.5), max_iters=30, early_stop=1),
    "gf32_n600_dv3_dc6": dict(q=32, n=600, dv=3, dc=6, code_seed=4103, data_seed=4203,
                              frames=4096, ebn0=(1.5, 3.5), max_iters=30, early_stop=1),
    "gf256_n128_dv2_dc8": dict(q=256, n=128, dv=2, dc=8, code_seed=4104, data_seed=4204,
                               frames=4096, ebn0=(1.5, 3.5), max_iters=30, early_stop=1),
}

# The mixed-code set decoded together: frame counts per code from a seeded
# lognormal with mean 4096 (sigma_ln = 1, mu = ln 4096 - 1/2, rounded, >= 1),
# per-frame Eb/N0 uniform in [1.5, 3.5) dB, up to 30 iterations.
MIXED_SET = ("gf16_n1024_dv2_dc4", "gf64_n576_dv2_dc4", "gf32_n600_dv3_dc6", "gf256_n128_dv2_dc8")
MIXED_EBN0 = (1.5, 3.5)
MIXED_SEED = 5151


def mixed_frame_counts(seed: int = MIXED_SEED) -> list[int]:
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = math.log(4096.0) - 0.5
    return [max(1, int(round(v))) for v in rng.lognormal(mu, 1.0, size=len(MIXED_SET))]


_CODE_CACHE: dict[str, Code] = {}


def workload_code(name: str) -> Code:
    if name not in _CODE_CACHE:
        w = WORKLOADS[name]
        _CODE_CACHE[name] = make_regular_code(w["q"], w["n"], w["dv"], w["dc"], w["code_seed"],
                                              name=name)
    return _CODE_CACHE[name]


def workload_seed(name: str, ebn0_index: int) -> int:
    return WORKLOADS[name]["data_seed"] * 1000 + 10 * ebn0_index
