"""One cluster over the ranks of a process group: the paper's domain
decomposition (section 3.2), parallel flow (section 3.3), sample sort
(section 3.4) and data redistribution (section 3.5), for a cluster larger
than one GPU's memory.

Each rank holds a contiguous block of the radially sorted stars: a multiple
of n_m = 20 stars on every rank but the last, which takes the rest (Eq. 17).
Bins of 20 stars and the relaxation pairs (2j, 2j + 1) then never straddle
two ranks, so the Eq. 7 timestep (up to a minimum over ranks) and the
relaxation run on each block alone.  Every rank also keeps the full sorted
radii and masses (section 3.2's duplicated arrays), from which it computes
the whole potential itself, without communication.

After the orbit step has moved the stars, the sorted order is rebuilt in
three exchanges:

1. Sample sort (section 3.4): each rank sorts its block by (r, id), takes s
   keys at evenly spaced positions, and all p s keys are gathered and sorted
   on every rank; the keys at positions s, 2s, ..., (p - 1) s of that list
   are the splitters.  Each rank cuts its block at the splitters (binary
   search), sends piece j to rank j (all-to-all) and sorts what it receives.
2. Redistribution (section 3.5): an exclusive prefix over the ranks' counts
   gives each rank the global positions of the stars it holds; the runs that
   Eq. 17 assigns to other ranks go there (all-to-all) and arrive in order.
3. The duplicated arrays: every rank gathers all radii and masses.

The collectives are torch.distributed's all_gather and all_to_all_single
(NCCL between GPUs, gloo between host processes); no GPU waits on another.
The per-rank compute (the local sort, the potential) is passed in; by
default it is the library's CUDA stage calls on device tensors.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

N_M = 20  # stars per rank are a multiple of this (the bin size), section 3.2

# fields of a star record exchanged by the sort, in one float64 row (ids
# below 2^53 are exact in a double)
FIELDS = ("r", "vr", "vt", "m", "id")


# ------------------------------------------------------------ partition
def partition_starts(n: int, p: int, n_m: int = N_M) -> list:
    """First global index of every rank's block and n (p + 1 entries):
    Eq. 17 with q = floor(n / n_m) blocks of n_m stars, floor(q / p) of
    them on every rank, one more on the first q mod p ranks, and the
    n - n_m q remaining stars on the last rank."""
    if n < 0 or p < 1 or n_m < 1:
        raise ValueError("partition_starts: n >= 0, p >= 1, n_m >= 1")
    q = n // n_m
    base, rem = q // p, q % p
    starts = [rank * base * n_m + min(rank, rem) * n_m for rank in range(p)]
    return starts + [n]


def global_index(i: int, rank: int, n: int, p: int, n_m: int = N_M) -> int:
    """Eq. 17: the global (sorted) index of local star i on rank `rank`."""
    q = n // n_m
    base, rem = q // p, q % p
    if rank < rem:
        return i + rank * base * n_m + rank * n_m
    return i + rank * base * n_m + rem * n_m


def redistribution_counts(held: list, n: int, p: int, n_m: int = N_M) -> list:
    """Section 3.5: send[j][d] = how many of the stars rank j holds (in
    global order, after the sample sort) belong to rank d's Eq. 17 block."""
    if sum(held) != n or len(held) != p:
        raise ValueError("redistribution_counts: held counts must sum to n over p ranks")
    starts = partition_starts(n, p, n_m)
    send = []
    before = 0
    for j in range(p):
        lo, hi = before, before + held[j]
        row = []
        for d in range(p):
            a, b = max(lo, starts[d]), min(hi, starts[d + 1])
            row.append(max(0, b - a))
        send.append(row)
        before = hi
    return send


# ----------------------------------------------------------- sample sort
def sample_positions(n_local: int, s: int) -> list:
    """s evenly spaced positions of a sorted block of n_local keys (the
    middles of s equal parts); fewer when the block is smaller."""
    if n_local <= 0 or s <= 0:
        return []
    s = min(s, n_local)
    return [((2 * k + 1) * n_local) // (2 * s) for k in range(s)]


def splitter_positions(n_samples: int, s: int, p: int) -> list:
    """Positions s, 2s, ..., (p - 1)s in the sorted list of all samples
    (clipped to the list)."""
    return [min(j * s, max(n_samples - 1, 0)) for j in range(1, p)]


def cut_points(r_sorted: torch.Tensor, id_sorted: torch.Tensor, split_r: torch.Tensor,
               split_id: torch.Tensor) -> list:
    """Offsets (p + 1) cutting a block sorted by (r, id) at the splitters:
    piece j holds the keys in [splitter_{j-1}, splitter_j)."""
    n = int(r_sorted.shape[0])
    out = [0]
    for j in range(int(split_r.shape[0])):
        sr, si = split_r[j], split_id[j]
        # first key not below the splitter: keys with r < sr, then the keys
        # with r == sr and id < si (a run ordered by id)
        lo = int(torch.searchsorted(r_sorted, sr.reshape(1), right=False)[0])
        hi = int(torch.searchsorted(r_sorted, sr.reshape(1), right=True)[0])
        if hi > lo:
            lo += int(torch.searchsorted(id_sorted[lo:hi].contiguous(), si.reshape(1),
                                         right=False)[0])
        out.append(max(lo, out[-1]))
    out.append(n)
    return out


def _default_local_sort(r: torch.Tensor, ids: torch.Tensor) -> torch.Tensor:
    """The library's key-value radix sort (cmc_sort_radius): the permutation
    that orders a block by (r, id)."""
    from . import stage_sort_radius
    return stage_sort_radius(r, ids).long()


def _default_potential(r: torch.Tensor, m: torch.Tensor) -> torch.Tensor:
    from . import stage_potential
    return stage_potential(r, m)


def _pack(rec: dict) -> torch.Tensor:
    cols = [rec[k].to(torch.float64) for k in FIELDS]
    return torch.stack(cols, dim=1).contiguous()


def _unpack(rows: torch.Tensor, like: dict) -> dict:
    out = {}
    for j, k in enumerate(FIELDS):
        col = rows[:, j].contiguous()
        out[k] = col.to(like[k].dtype) if like[k].dtype != torch.float64 else col
    return out


class ShardedCluster:
    """The sorted state of one cluster spread over the ranks of `group`
    (default: the world), this rank's block plus the duplicated radii and
    masses.  `local_sort(r, ids) -> permutation` and `potential(r, m) -> Phi`
    run the per-rank work (default: the library's kernels)."""

    def __init__(self, n_total: int, group=None, samples_per_rank: int = 64,
                 local_sort=None, potential=None):
        self.group = group
        self.p = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.n = int(n_total)
        self.s = int(samples_per_rank)
        self.local_sort = local_sort or _default_local_sort
        self.potential = potential or _default_potential
        self.starts = partition_starts(self.n, self.p)

    # -------------------------------------------------------------- sort
    def _sorted(self, rec: dict) -> dict:
        if rec["r"].shape[0] == 0:
            return rec
        perm = self.local_sort(rec["r"], rec["id"])
        return {k: v[perm] for k, v in rec.items()}

    def _all_gather_varlen(self, t: torch.Tensor) -> list:
        """Tensors of different lengths (first dimension) from every rank."""
        n_here = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
        sizes = [torch.zeros_like(n_here) for _ in range(self.p)]
        dist.all_gather(sizes, n_here, group=self.group)
        sizes = [int(x.item()) for x in sizes]
        width = max(sizes) if sizes else 0
        pad = torch.zeros((width,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[: t.shape[0]] = t
        bufs = [torch.empty_like(pad) for _ in range(self.p)]
        dist.all_gather(bufs, pad, group=self.group)
        return [b[:k] for b, k in zip(bufs, sizes)]

    def _exchange(self, rows: torch.Tensor, send: list) -> torch.Tensor:
        """All-to-all of row blocks: send[d] rows (in order) to rank d."""
        n_send = torch.tensor(send, dtype=torch.int64, device=rows.device)
        n_recv = torch.empty_like(n_send)
        dist.all_to_all_single(n_recv, n_send, group=self.group)
        recv = [int(x) for x in n_recv.tolist()]
        out = torch.empty((sum(recv), rows.shape[1]), dtype=rows.dtype, device=rows.device)
        dist.all_to_all_single(out, rows, output_split_sizes=recv, input_split_sizes=send,
                               group=self.group)
        return out

    def sort(self, rec: dict) -> dict:
        """This rank's stars after a step (any radii, any order, any count)
        -> this rank's Eq. 17 block of the globally (r, id)-sorted stars."""
        rec = self._sorted(rec)
        n_local = int(rec["r"].shape[0])
        # samples and splitters (phases 2 and 3)
        pos = torch.tensor(sample_positions(n_local, self.s), dtype=torch.long,
                           device=rec["r"].device)
        samp = torch.stack([rec["r"][pos].to(torch.float64),
                            rec["id"][pos].to(torch.float64)], dim=1)
        allsamp = torch.cat(self._all_gather_varlen(samp), dim=0)
        if allsamp.shape[0]:
            order = self.local_sort(allsamp[:, 0].contiguous(),
                                    allsamp[:, 1].to(rec["id"].dtype).contiguous())
            allsamp = allsamp[order]
        sp = splitter_positions(int(allsamp.shape[0]), self.s, self.p)
        if allsamp.shape[0]:
            split_r = allsamp[sp, 0]
            split_id = allsamp[sp, 1].to(rec["id"].dtype)
        else:
            split_r = torch.zeros(0, dtype=torch.float64, device=rec["r"].device)
            split_id = torch.zeros(0, dtype=rec["id"].dtype, device=rec["r"].device)
        # exchange the pieces (phase 4) and sort what arrived (phase 5)
        cuts = cut_points(rec["r"], rec["id"], split_r, split_id)
        send = [cuts[j + 1] - cuts[j] for j in range(self.p)]
        got = _unpack(self._exchange(_pack(rec), send), rec)
        got = self._sorted(got)
        # redistribution to the Eq. 17 blocks (section 3.5)
        held = torch.tensor([got["r"].shape[0]], dtype=torch.int64, device=got["r"].device)
        counts = [torch.zeros_like(held) for _ in range(self.p)]
        dist.all_gather(counts, held, group=self.group)
        plan = redistribution_counts([int(c.item()) for c in counts], self.n, self.p)
        block = _unpack(self._exchange(_pack(got), plan[self.rank]), got)
        assert block["r"].shape[0] == self.starts[self.rank + 1] - self.starts[self.rank]
        return block

    # --------------------------------------------------- duplicated arrays
    def gather_rm(self, block: dict):
        """Every rank's copy of all radii and masses (in global order)."""
        r = torch.cat(self._all_gather_varlen(block["r"]), dim=0)
        m = torch.cat(self._all_gather_varlen(block["m"]), dim=0)
        return r, m

    def local_potential(self, block: dict):
        """Phi of this rank's stars, from the full duplicated arrays: the
        potential of the bound stars (finite r) computed on every rank, the
        same on all of them, then this rank's part."""
        r, m = self.gather_rm(block)
        nb = int(torch.isfinite(r).sum().item())
        phi = torch.zeros_like(r)
        if nb:
            phi[:nb] = self.potential(r[:nb].contiguous(), m[:nb].contiguous())
        a, b = self.starts[self.rank], self.starts[self.rank + 1]
        return phi[a:b], phi
