"""Gallery sharding by pack across the GPUs of one node.

The paper's cluster architecture (Sec. 3.4) splits the gallery over clusters: the
main server sends each cluster the encrypted query and combines the clusters'
outputs with the compression method.  Here a rank (one GPU) plays a cluster.  The
unit of a shard is a pack -- the s consecutive groups whose HE-C^3 outputs the
compression puts into one score ciphertext (a group when the layout has no
compression) -- so no compression crosses two shards, and the score ciphertexts of
the shards, concatenated in rank order, are those of the unsharded match.  Every
rank encodes its own identities, runs Algorithm 1 on the same query itself
(recomputing it is cheaper than sending the N_in expanded ciphertexts) and its
match; rank 0 gathers the score ciphertexts (host buffers through the process
group: a few MiB per query).  This module holds only the partition and the gather;
the match is the library's.
"""
import numpy as np


def ids_per_unit(slots, part, complex_pack, compressed):
    """Identities of one output unit: a group holds slots/part identities (twice
    that with complex packing), a pack s = part groups."""
    per_group = (2 if complex_pack else 1) * slots // part
    return per_group * part if compressed else per_group


def shard_range(n_ids, slots, part, complex_pack, compressed, rank, world):
    """[lo, hi) identities of rank's shard: whole units, split as evenly as the
    unit count allows (empty for the ranks beyond it)."""
    u = ids_per_unit(slots, part, complex_pack, compressed)
    n_units = -(-n_ids // u)
    u0, u1 = rank * n_units // world, (rank + 1) * n_units // world
    return min(u0 * u, n_ids), min(u1 * u, n_ids)


def gather_outputs(local, rank, world):
    """Rank 0 receives every rank's score ciphertexts ([queries][units][...] uint64,
    or None for an empty shard) and returns them concatenated along the unit axis in
    rank order; the other ranks return None.  world == 1: local itself."""
    if world == 1:
        return local
    import torch.distributed as dist
    parts = [None] * world if rank == 0 else None
    dist.gather_object(local, parts, dst=0)
    if rank != 0:
        return None
    return np.concatenate([p for p in parts if p is not None], axis=1)
