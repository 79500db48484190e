"""Synthetic similarity graphs and starting memberships.

Every draw comes from the counter-based generator in :mod:`synth.rng`, and
everything that decides an edge is integer arithmetic, so a graph drawn on a
CUDA device is bit-identical to the same graph drawn on the CPU.  The only
floating-point step that shapes a graph (the Pareto degree propensities) is
always evaluated on the CPU.

Graph families
--------------
* ``sbm_pairs``: planted-partition SBM by independent Bernoulli trials over
  all pairs (O(n^2), small n only).
* ``dcsbm_edges``: degree-corrected SBM with power-law propensities and
  overlapping blocks, drawn edge by edge (O(edges)); nodes are relabelled by a
  seeded permutation so that row order carries no locality.  This stands in
  for citation graphs such as the paper's Web of Science and OpenAlex sets
  (Sect. 5), reproducing their scale and heavy-tailed degrees, not their
  records.
* ``two_cluster_er_edges``: two Erdos-Renyi clusters joined by a fixed number
  of bridges, the paper's artificial graph (Sect. 5, "Artificial graph").

``assemble_csr`` turns an undirected edge list into the symmetric similarity
matrix of the paper's construction (Example 4.1 and Sect. 5
"Hyperparameters"): s_ij = s_ji for every edge, ones on the diagonal.  Edge
weights are a pure function of the unordered pair, so duplicate edges carry
equal weights.
"""
from __future__ import annotations

import dataclasses
import math

import torch

from .rng import bits_below, below, hash_u64, uniform01

# stream identifiers: one independent counter space per kind of draw
_S_PAIR, _S_WEIGHT, _S_NBLK, _S_B0, _S_B1, _S_B2, _S_THETA = 1, 2, 3, 4, 5, 6, 7
_S_EI, _S_EIN, _S_ESLOT, _S_EJB, _S_EJG, _S_PERM, _S_U0 = 8, 9, 10, 11, 12, 13, 14
_S_ER1, _S_ER2, _S_BRIDGE = 15, 16, 17


def _dev(device) -> torch.device:
    return torch.device(device) if device is not None else torch.device("cpu")


# ----------------------------------------------------------------------------
# weights
# ----------------------------------------------------------------------------
def pair_weights(a: torch.Tensor, b: torch.Tensor, n: int, seed: int) -> torch.Tensor:
    """Weight in (0, 1] of the undirected pair {a, b}: 1 - m * 2^-24 with m the
    top 24 bits of a draw keyed by (min, max).  Exactly representable in fp32."""
    lo = torch.minimum(a, b).to(torch.int64)
    hi = torch.maximum(a, b).to(torch.int64)
    m = bits_below(hash_u64(seed, _S_WEIGHT, lo * n + hi), 24)
    return (1.0 - m.to(torch.float64) * (2.0 ** -24)).to(torch.float32)


# ----------------------------------------------------------------------------
# planted-partition SBM over all pairs
# ----------------------------------------------------------------------------
def sbm_pairs(n: int, blocks: int, p_in: float, p_out: float, seed: int,
              device=None) -> tuple[torch.Tensor, torch.Tensor]:
    """Undirected edges (i < j) of an SBM with ``blocks`` equal blocks (node i in
    block i // (n // blocks)); each pair is an edge independently with
    probability p_in inside a block and p_out across blocks."""
    dev = _dev(device)
    size = n // blocks
    iu = torch.triu_indices(n, n, offset=1, device=dev)
    i, j = iu[0].to(torch.int64), iu[1].to(torch.int64)
    same = (i // size) == (j // size)
    thr_in = int(p_in * (1 << 53))
    thr_out = int(p_out * (1 << 53))
    draw = bits_below(hash_u64(seed, _S_PAIR, i * n + j), 53)
    keep = torch.where(same, draw < thr_in, draw < thr_out)
    return i[keep], j[keep]


# ----------------------------------------------------------------------------
# degree-corrected SBM with power-law propensities
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class _NodeTables:
    n: int
    nblk: torch.Tensor        # [n] blocks per node (1..3)
    blk: torch.Tensor         # [n, 3] block ids (entries past nblk unused)
    cdf: torch.Tensor         # [n] inclusive cumulative integer propensity
    total: int
    mem_cdf: torch.Tensor     # [sum nblk] cumulative propensity over (block, node)-sorted memberships
    mem_node: torch.Tensor    # [sum nblk] node of each membership
    blk_base: torch.Tensor    # [B] mem_cdf value before the block's first member
    blk_w: torch.Tensor       # [B] block's total propensity
    theta_max: float


def _node_tables(n: int, blocks: int, gamma: float, seed: int, device=None) -> _NodeTables:
    """Per-node memberships and integer propensities.  The Pareto draw (the
    only floating-point step) is always evaluated on the CPU; the integer
    tables are built on ``device`` (integer results do not depend on it)."""
    dev = _dev(device)
    B = blocks
    # Pareto(alpha = gamma - 1, x_min = 1) propensities, capped at sqrt(sum)
    alpha = gamma - 1.0
    u = uniform01(seed, _S_THETA, torch.arange(n, dtype=torch.int64))
    theta = torch.pow(u, -1.0 / alpha)
    del u
    cap = math.sqrt(float(theta.sum()))
    theta = torch.clamp(theta, max=cap)
    theta_max = float(theta.max())
    w = torch.floor(theta * 65536.0).to(torch.int64).to(dev)
    del theta
    idx = torch.arange(n, dtype=torch.int64, device=dev)
    nblk = torch.clamp(1 + below(seed, _S_NBLK, idx, 3), max=B)
    b0 = below(seed, _S_B0, idx, B)
    blk = torch.zeros((n, 3), dtype=torch.int64, device=dev)
    blk[:, 0] = b0
    if B >= 2:
        off1 = 1 + below(seed, _S_B1, idx, B - 1)
        blk[:, 1] = (b0 + off1) % B
        if B >= 3:
            off2 = 1 + below(seed, _S_B2, idx, B - 2)
            off2 = torch.where(off2 >= off1, off2 + 1, off2)
            blk[:, 2] = (b0 + off2) % B
            del off2
        del off1
    del b0
    cdf = torch.cumsum(w, 0)
    total = int(cdf[-1])
    # memberships sorted by (block, node)
    slot = torch.arange(3, dtype=torch.int64, device=dev).unsqueeze(0).expand(n, 3)
    valid = slot < nblk.unsqueeze(1)
    mb = blk[valid]
    mn = idx.unsqueeze(1).expand(n, 3)[valid]
    del valid, idx
    order = torch.argsort(mb * n + mn)
    mb, mn = mb[order], mn[order]
    del order
    mem_cdf = torch.cumsum(w[mn], 0)
    counts = torch.bincount(mb, minlength=B)
    del mb
    ends = torch.cumsum(counts, 0)
    starts = ends - counts
    blk_base = torch.where(starts > 0, mem_cdf[torch.clamp(starts - 1, min=0)], torch.zeros_like(starts))
    blk_end = torch.where(counts > 0, mem_cdf[torch.clamp(ends - 1, min=0)], blk_base)
    blk_w = blk_end - blk_base
    return _NodeTables(n, nblk, blk, cdf, total, mem_cdf, mn, blk_base, blk_w, theta_max)


def dcsbm_edges(n: int, blocks: int, mean_deg: float, seed: int, gamma: float = 2.5,
                mu_in: float = 0.8, device=None, chunk: int = 1 << 25,
                relabel: bool = True) -> tuple[torch.Tensor, torch.Tensor]:
    """Undirected edge list of a degree-corrected SBM.

    * node i joins 1-3 distinct blocks of ``blocks``;
    * propensity theta_i ~ Pareto(gamma - 1, 1), capped at sqrt(sum theta);
    * E = n (mean_deg - 1) / 2 edges: endpoint i drawn with probability
      proportional to theta; with probability ``mu_in`` the other endpoint is
      drawn proportional to theta inside one of i's blocks, otherwise over all
      nodes;
    * nodes are then relabelled by a seeded random permutation.

    Self-loops and duplicates are left in; :func:`assemble_csr` drops and
    merges them, so the matrix has slightly fewer than ``n * mean_deg``
    nonzeros.  Returned tensors are int64 on ``device``.
    """
    dev = _dev(device)
    t = _node_tables(n, blocks, gamma, seed, dev)
    cdf, nblk, blk, mem_cdf, mem_node, blk_base, blk_w = (
        t.cdf, t.nblk, t.blk, t.mem_cdf, t.mem_node, t.blk_base, t.blk_w)
    E = int(round(n * (mean_deg - 1.0) / 2.0))
    thr_in = int(mu_in * (1 << 20))
    if relabel:
        perm_key = hash_u64(seed, _S_PERM, torch.arange(n, dtype=torch.int64, device=dev))
        order = torch.argsort(perm_key, stable=True)
        perm = torch.empty(n, dtype=torch.int64, device=dev)
        perm[order] = torch.arange(n, dtype=torch.int64, device=dev)
        del perm_key, order
    srcs, dsts = [], []
    for e0 in range(0, E, chunk):
        e = torch.arange(e0, min(E, e0 + chunk), dtype=torch.int64, device=dev)
        i = torch.searchsorted(cdf, below(seed, _S_EI, e, t.total), right=True)
        inb = bits_below(hash_u64(seed, _S_EIN, e), 20) < thr_in
        slot = below(seed, _S_ESLOT, e, nblk[i])
        b = blk[i, slot]
        wb = blk_w[b]
        rj = below(seed, _S_EJB, e, torch.clamp(wb, min=1))
        jb = mem_node[torch.searchsorted(mem_cdf, blk_base[b] + rj, right=True)]
        jg = torch.searchsorted(cdf, below(seed, _S_EJG, e, t.total), right=True)
        j = torch.where(inb & (wb > 0), jb, jg)
        if relabel:
            i, j = perm[i], perm[j]
        srcs.append(i)
        dsts.append(j)
    if not srcs:
        z = torch.zeros(0, dtype=torch.int64, device=dev)
        return z, z.clone()
    return torch.cat(srcs), torch.cat(dsts)


# ----------------------------------------------------------------------------
# two Erdos-Renyi clusters joined by bridges (paper Sect. 5, artificial graph)
# ----------------------------------------------------------------------------
def two_cluster_er_edges(n1: int, n2: int, p1: float, p2: float, bridges: int, seed: int,
                         device=None, chunk: int = 1 << 25) -> tuple[torch.Tensor, torch.Tensor]:
    """Cluster 1 = nodes [0, n1), cluster 2 = [n1, n1 + n2).  Each cluster gets
    round(p * c (c - 1) / 2) uniformly drawn node pairs (a G(n, m) stand-in for
    G(n, p) at sizes where all-pairs trials are out of reach); ``bridges``
    pairs join the clusters.  Self-loops and duplicates are merged later."""
    dev = _dev(device)
    out_s, out_d = [], []
    for (base, c, p, stream) in ((0, n1, p1, _S_ER1), (n1, n2, p2, _S_ER2)):
        m = int(round(p * c * (c - 1) / 2.0))
        for e0 in range(0, m, chunk):
            e = torch.arange(e0, min(m, e0 + chunk), dtype=torch.int64, device=dev)
            a = below(seed, stream, 2 * e, c)
            b = below(seed, stream, 2 * e + 1, c)
            out_s.append(a + base)
            out_d.append(b + base)
    e = torch.arange(bridges, dtype=torch.int64, device=dev)
    out_s.append(below(seed, _S_BRIDGE, 2 * e, n1))
    out_d.append(n1 + below(seed, _S_BRIDGE, 2 * e + 1, n2))
    return torch.cat(out_s), torch.cat(out_d)


def two_cluster_graph(n1: int, n2: int, deg1: float, deg2: float, bridges: int, seed: int,
                      device=None, weighted: bool = False):
    """The paper's artificial graph (Sect. 5, "Artificial graph"): two
    Erdos-Renyi clusters of n1 and n2 nodes with edge probabilities
    deg1 / (n1 - 1) and deg2 / (n2 - 1), ``bridges`` random inter-cluster edges,
    0/1 similarity (unless ``weighted``) with a unit diagonal.  The paper's run
    uses n1 = 500,000, n2 = 250,000, deg1 = 1200, deg2 = 1600, 200 bridges.
    The paper prunes nodes of degree 0; at these degrees none occurs (checked).
    Returns (row_ptr, col, val, labels) with labels 0 on [0, n1), 1 after."""
    n = n1 + n2
    s, d = two_cluster_er_edges(n1, n2, deg1 / (n1 - 1), deg2 / (n2 - 1), bridges, seed, device=device)
    rp, c, v = assemble_csr(n, s, d, seed, weighted=weighted)
    if n > 0 and int((rp[1:] - rp[:-1]).min()) < 2:
        raise ValueError("a node without edges: the paper's pruning would remove it")
    labels = torch.zeros(n, dtype=torch.int64, device=rp.device)
    labels[n1:] = 1
    return rp, c, v, labels


def second_row_start(n: int, k: int = 2, device=None) -> torch.Tensor:
    """The artificial-graph experiment's start X^0: every article fully in the
    second cluster (U0 = e_2 in every row)."""
    U0 = torch.zeros((n, k), dtype=torch.float32, device=_dev(device))
    U0[:, 1] = 1.0
    return U0


# ----------------------------------------------------------------------------
# CSR assembly
# ----------------------------------------------------------------------------
def assemble_csr(n: int, src: torch.Tensor, dst: torch.Tensor, seed: int,
                 max_chunk_entries: int = 1 << 29,
                 weighted: bool = True) -> tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """Symmetric CSR of the similarity matrix: for each edge {a, b} with a != b,
    s_ab = s_ba = pair_weights(a, b) (or 1 when ``weighted`` is false, the
    paper's 0/1 citation similarity); duplicates merge (equal weights); s_ii = 1.

    Returns (row_ptr int64 [n+1], col int32 [nnz], val float32 [nnz]) on the
    device of ``src``.  Columns are sorted within each row.  Rows are built in
    chunks so that no sort exceeds ``max_chunk_entries`` keys.
    """
    dev = src.device
    src = src.to(torch.int64)
    dst = dst.to(torch.int64)
    nz = src != dst
    src, dst = src[nz], dst[nz]
    deg = torch.bincount(src, minlength=n) + torch.bincount(dst, minlength=n) + 1
    cum = torch.cumsum(deg, 0)
    # row-chunk boundaries so that each chunk holds at most max_chunk_entries keys
    bounds = [0]
    total = int(cum[-1]) if n > 0 else 0
    target = max_chunk_entries
    while bounds[-1] < n:
        prev = int(cum[bounds[-1] - 1]) if bounds[-1] > 0 else 0
        nxt = int(torch.searchsorted(cum, torch.tensor(prev + target, device=dev), right=True))
        nxt = max(nxt, bounds[-1] + 1)
        bounds.append(min(nxt, n))
    del cum, deg
    cols, vals, counts = [], [], []
    for r0, r1 in zip(bounds[:-1], bounds[1:]):
        m1 = (src >= r0) & (src < r1)
        m2 = (dst >= r0) & (dst < r1)
        rows = torch.arange(r0, r1, dtype=torch.int64, device=dev)
        keys = torch.cat([src[m1] * n + dst[m1], dst[m2] * n + src[m2], rows * n + rows])
        del m1, m2
        keys = torch.unique(keys, sorted=True)
        r = keys // n
        c = keys % n
        if weighted:
            w = pair_weights(r, c, n, seed)
            w = torch.where(r == c, torch.ones_like(w), w)
        else:
            w = torch.ones(r.shape, dtype=torch.float32, device=dev)
        cols.append(c.to(torch.int32))
        vals.append(w)
        counts.append(torch.bincount(r - r0, minlength=r1 - r0))
        del keys, r, c
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    if n > 0:
        row_ptr[1:] = torch.cumsum(torch.cat(counts), 0)
    col = torch.cat(cols) if cols else torch.zeros(0, dtype=torch.int32, device=dev)
    val = torch.cat(vals) if vals else torch.zeros(0, dtype=torch.float32, device=dev)
    assert total >= col.numel()
    return row_ptr, col, val


# ----------------------------------------------------------------------------
# starting memberships
# ----------------------------------------------------------------------------
def dirichlet_u0(n: int, k: int, seed: int, device=None, chunk_rows: int = 1 << 22) -> torch.Tensor:
    """Rows ~ Dirichlet(1): e_ia = -ln(u_ia), u in (0, 1], normalised per row in
    float64 and stored as float32 (n x k, row-major)."""
    dev = _dev(device)
    out = torch.empty((n, k), dtype=torch.float32, device=dev)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        idx = torch.arange(r0 * k, r1 * k, dtype=torch.int64, device=dev)
        e = -torch.log(uniform01(seed, _S_U0, idx)).view(r1 - r0, k)
        out[r0:r1] = (e / e.sum(dim=1, keepdim=True)).to(torch.float32)
    return out


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class GraphSpec:
    """A named synthetic workload: graph family, size, clusters and seed."""
    kind: str                 # "sbm" | "dcsbm" | "er2"
    n: int
    k: int
    seed: int
    mean_deg: float = 30.0
    blocks: int = 0           # 0 -> k
    p_in: float = 0.02
    p_out: float = 0.001
    gamma: float = 2.5

    @property
    def nblocks(self) -> int:
        return self.blocks if self.blocks > 0 else self.k


def make_graph(spec: GraphSpec, device=None):
    """(row_ptr, col, val) of the workload's similarity matrix on ``device``."""
    dev = _dev(device)
    if spec.kind == "sbm":
        s, d = sbm_pairs(spec.n, spec.nblocks, spec.p_in, spec.p_out, spec.seed, device=dev)
    elif spec.kind == "dcsbm":
        s, d = dcsbm_edges(spec.n, spec.nblocks, spec.mean_deg, spec.seed, gamma=spec.gamma, device=dev)
    else:
        raise ValueError(f"unknown graph kind {spec.kind}")
    return assemble_csr(spec.n, s, d, spec.seed)


def batch_specs(count: int, seed: int = 3, n_range=(500, 200_000), ks=(4, 8, 16, 32, 64),
                deg_range=(10.0, 40.0)) -> list:
    """Instances of a batched workload: n log-uniform in n_range, k uniform
    over ks, mean degree uniform in deg_range, DC-SBM graphs with B = k blocks
    and seed + b per instance (draws from the same counter-based generator)."""
    idx = torch.arange(count, dtype=torch.int64)
    un = uniform01(seed, 101, idx).numpy()
    uk = below(seed, 102, idx, len(ks)).numpy()
    ud = uniform01(seed, 103, idx).numpy()
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    out = []
    for b in range(count):
        n = int(round(math.exp(lo + (hi - lo) * (1.0 - un[b]))))
        k = int(ks[int(uk[b])])
        d = deg_range[0] + (deg_range[1] - deg_range[0]) * (1.0 - ud[b])
        out.append(GraphSpec("dcsbm", n, k, seed + b, mean_deg=d))
    return out
