"""Sharding a multi-domain batch across GPUs (host logic, no arithmetic of the method).

A multi-domain evolution holds many grids of uneven point counts (Sec. 1). The points of different
grids are independent, so the grids can be spread over several GPUs with no exchange between them. Each
GPU then runs its share as one batched launch. The share is chosen by the longest-processing-time rule:
grids in decreasing size, each to the GPU with the fewest points so far. The largest share is then at
most the average share plus the largest single grid.
"""


def lpt_partition(sizes, parts):
    """Indices of `sizes` split into `parts` lists by the longest-processing-time rule.

    Deterministic: ties in size go to the lower index first, and ties in load to the lower part. Each
    list is returned in ascending index order. Every index appears in exactly one list; with more parts
    than sizes, some lists are empty.
    """
    if parts < 1:
        raise ValueError("parts must be >= 1")
    sizes = [int(s) for s in sizes]
    if any(s < 0 for s in sizes):
        raise ValueError("sizes must be >= 0")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * parts
    out = [[] for _ in range(parts)]
    for i in order:
        p = min(range(parts), key=lambda q: (load[q], q))
        out[p].append(i)
        load[p] += sizes[i]
    return [sorted(o) for o in out]
