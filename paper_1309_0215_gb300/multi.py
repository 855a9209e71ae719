"""Sharding a job over several GPUs and merging the per-GPU results (host side).

The map/reduce path shards naturally (arXiv:1309.0215 Sec. II-A: the input
is cut into independent splits, and the intermediate pairs are partitioned
by key for the reduce): each rank runs the job on its own slice with the
single-GPU library, then

* array containers (RGB histogram, regression sums, large-key histogram)
  are combined with one all-reduce (sum) of the container, and Bloom
  filters with a bitwise OR of their bit arrays;
* word count is combined in the paper's partition step: every rank sends
  each of its (key, count) records to the rank that owns the key's hash
  partition (one all-to-all), each rank adds up the counts of its partition
  and sorts it, and rank 0 merges the sorted partitions (k-way) into the
  result layout of include/mr.h.

Slices are cut where no work unit straddles two of them: on a multiple of 3
bytes (pixels), 2 bytes (pairs) or 4 bytes (keys), and for text just after
an ASCII whitespace byte, so every token lies in exactly one slice.  A
Bloom job's slices own the windows that start in them and overlap the next
slice by one window less a base, so every window lies whole in exactly one
slice.

The functions here move and reorder results between ranks; the map and
combine work itself runs in the library's kernels on each rank.  The merge
is written for torch.distributed (any backend that has all_to_all_single
and gather_object: gloo on CPU ranks, NCCL with CUDA tensors).  k-means is
not sharded here: its per-iteration K x D sums would have to be exchanged
inside a job, and a job runs all its iterations in one call.
"""
import heapq
import zlib

import numpy as np

from . import BLOOM_DNA, HIST_RGB8, HIST_U32, LINREG_I8, WORDCOUNT

_WS = frozenset(b" \t\n\v\f\r")


def _whitespace_at_or_after(read, n, pos):
    """First index >= pos whose byte is ASCII whitespace (n if none);
    read(lo, hi) returns bytes [lo, hi) of the input."""
    step = 4096
    while pos < n:
        hi = min(n, pos + step)
        chunk = read(pos, hi)
        for i, b in enumerate(chunk):
            if b in _WS:
                return pos + i
        pos = hi
        step *= 2
    return n


def shard_bounds(kind, n, world, rank, read=None, kmer=None):
    """Byte range [lo, hi) of rank's slice of an n-byte input.

    kind: HIST_RGB8 (slices of whole pixels), LINREG_I8 (whole pairs),
    HIST_U32 (whole 4-byte keys), WORDCOUNT (each boundary moved forward to
    the next whitespace byte, so no token is cut; read(lo, hi) must return
    input bytes [lo, hi)) or BLOOM_DNA (kmer: the window length; the slice
    holds the windows that start in rank's share of the positions, so it
    runs kmer - 1 bytes into the next share).  Except for BLOOM_DNA, the
    slices of ranks 0 .. world-1 cover [0, n) without overlap."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world size or rank")
    if kind == BLOOM_DNA:
        if not kmer or kmer < 1:
            raise ValueError("a Bloom job needs its window length")
        lo, hi = n * rank // world, n * (rank + 1) // world
        return lo, min(n, hi + kmer - 1)
    if kind in (HIST_RGB8, LINREG_I8, HIST_U32):
        unit = {HIST_RGB8: 3, LINREG_I8: 2, HIST_U32: 4}[kind]
        if n % unit:
            raise ValueError("input length is not a multiple of the record size")
        units = n // unit
        return unit * (units * rank // world), unit * (units * (rank + 1) // world)
    if kind != WORDCOUNT:
        raise ValueError("kind is not sharded by byte ranges")
    if read is None:
        raise ValueError("word count needs read(lo, hi) to find token boundaries")

    def cut(r):
        return 0 if r == 0 else (n if r == world else _whitespace_at_or_after(read, n, n * r // world))
    return cut(rank), cut(rank + 1)


def reader(data):
    """read(lo, hi) over a bytes object, a numpy uint8 array or a torch uint8
    tensor (a device tensor is read in small windows)."""
    if isinstance(data, (bytes, bytearray, memoryview)):
        return lambda lo, hi: bytes(data[lo:hi])
    if isinstance(data, np.ndarray):
        return lambda lo, hi: data[lo:hi].tobytes()
    return lambda lo, hi: data[lo:hi].cpu().numpy().tobytes()


def allreduce_sum(t, group=None):
    """Sum an array container (768 histogram bins, the five regression sums or
    a large-key histogram's bins; int64) over all ranks, in place; returns t."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def allreduce_or(t, group=None):
    """Bitwise OR of a Bloom filter's bit array (uint8) over all ranks, in
    place; returns t.  The ranks' arrays are gathered and ORed where t lives
    (NCCL has no bitwise reduction)."""
    import torch
    import torch.distributed as dist
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    for p in parts:
        t.bitwise_or_(p)
    return t


def merge_bloom_local(arrays):
    """The whole input's Bloom filter from its slices' filters, in one process."""
    out = np.zeros_like(np.asarray(arrays[0], dtype=np.uint8))
    for a in arrays:
        out |= np.asarray(a, dtype=np.uint8)
    return out


# ---------------------------------------------------------------- word count
# Result layout (include/mr.h): u64 records, u64 key bytes, then per record
# u64 {count, key offset, key length}, then the concatenated keys; records
# ordered by count descending, then key bytes ascending.

def wordcount_records(blob):
    """[(key bytes, count), ...] of a word-count result."""
    n, kb = (int(v) for v in np.frombuffer(blob[:16], dtype=np.uint64))
    rec = np.frombuffer(blob[16:16 + 24 * n], dtype=np.uint64).reshape(n, 3)
    keys = bytes(blob[16 + 24 * n:16 + 24 * n + kb])
    return [(keys[int(o):int(o) + int(l)], int(c)) for c, o, l in rec]


def wordcount_blob(records):
    """The result layout of already ordered [(key, count), ...]."""
    n = len(records)
    rec = np.empty((n, 3), dtype=np.uint64)
    off = 0
    for i, (k, c) in enumerate(records):
        rec[i] = (c, off, len(k))
        off += len(k)
    head = np.array([n, off], dtype=np.uint64).tobytes()
    return head + rec.tobytes() + b"".join(k for k, _ in records)


def _order(item):
    return (-item[1], item[0])


def partition_of(key, world):
    """The rank that reduces a key: its CRC-32 modulo the number of ranks
    (the same on every process, unlike Python's salted hash)."""
    return zlib.crc32(key) % world


def reduce_partition(parts):
    """Add up the counts of equal keys over record lists and order them."""
    acc = {}
    for recs in parts:
        for k, c in recs:
            acc[k] = acc.get(k, 0) + c
    return sorted(acc.items(), key=_order)


def kway_merge(sorted_parts):
    """Merge partitions that are each ordered and hold disjoint keys."""
    return list(heapq.merge(*sorted_parts, key=_order))


def merge_wordcount_local(blobs):
    """The whole-input result from the slices' results, in one process (the
    same partition, reduce and k-way merge steps as merge_wordcount)."""
    world = max(1, len(blobs))
    parts = [[] for _ in range(world)]
    for blob in blobs:
        for k, c in wordcount_records(blob):
            parts[partition_of(k, world)].append((k, c))
    return wordcount_blob(kway_merge([reduce_partition([p]) for p in parts]))


def merge_wordcount(blob, group=None, device=None):
    """Combine the ranks' word-count results of their slices.  Every rank
    calls this with its own result; rank 0 gets the whole input's result in
    the layout of include/mr.h, the other ranks None.

    The records go to their key's partition with one all-to-all of byte
    buffers (device: where the exchanged tensors live, e.g. "cuda" for NCCL;
    CPU for gloo), each rank reduces its partition, and rank 0 gathers the
    ordered partitions and merges them k-way."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    out = [[] for _ in range(world)]
    for k, c in wordcount_records(blob):
        out[partition_of(k, world)].append((k, c))
    send = [np.frombuffer(wordcount_blob(p), dtype=np.uint8) for p in out]
    sizes = torch.tensor([len(b) for b in send], dtype=torch.int64, device=device)
    rsizes = torch.empty(world, dtype=torch.int64, device=device)
    dist.all_to_all_single(rsizes, sizes, group=group)
    rs = [int(v) for v in rsizes.cpu()]
    sbuf = torch.from_numpy(np.concatenate(send)).to(device) if send else torch.empty(0, dtype=torch.uint8)
    rbuf = torch.empty(sum(rs), dtype=torch.uint8, device=device)
    dist.all_to_all_single(rbuf, sbuf, output_split_sizes=rs, input_split_sizes=[len(b) for b in send], group=group)
    raw = rbuf.cpu().numpy().tobytes()
    mine, pos = [], 0
    for sz in rs:
        mine.append(wordcount_records(raw[pos:pos + sz]))
        pos += sz
    part = reduce_partition(mine)
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(part, gathered, dst=0, group=group)
    if rank != 0:
        return None
    return wordcount_blob(kway_merge(gathered))
