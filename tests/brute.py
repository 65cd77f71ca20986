"""Brute-force explicit de Bruijn graph, for pinning the oracle on tiny inputs.

Independent of ``oracle/``: it builds G(S, k) literally as Python sets of
k-mer and (k+1)-mer strings (section "Preliminaries"), adds the reverse
complements for the comprehensive graph (paragraph after Algorithm 2), and
compacts it by walking maximal non-branching paths, the "naive compaction
algorithm" the paper checks its output against (Results section).
"""
from collections import defaultdict
from typing import Dict, Iterable, List, Set, Tuple

_TR = str.maketrans("ACGT", "TGCA")


def revcomp(s: str) -> str:
    return s.translate(_TR)[::-1]


def texts(strings: Iterable[str], both: bool) -> List[str]:
    strings = list(strings)
    return strings + ([revcomp(s) for s in strings] if both else [])


def graph(strings: Iterable[str], k: int, both: bool):
    """(vertices, edges, sentinels) of G(S, k), or of the comprehensive graph."""
    V: Set[str] = set()
    E: Set[str] = set()
    sentinels: Set[str] = set()
    for t in texts(strings, both):
        for i in range(len(t) - k + 1):
            V.add(t[i:i + k])
        for i in range(len(t) - k):
            E.add(t[i:i + k + 1])
        if len(t) >= k:
            sentinels.add(t[:k])
            sentinels.add(t[-k:])
    return V, E, sentinels


def junction_kmers(strings: Iterable[str], k: int, both: bool) -> Set[str]:
    V, E, sentinels = graph(strings, k, both)
    indeg: Dict[str, int] = defaultdict(int)
    outdeg: Dict[str, int] = defaultdict(int)
    for e in E:
        outdeg[e[:-1]] += 1
        indeg[e[1:]] += 1
    return {v for v in V if v in sentinels or indeg[v] > 1 or outdeg[v] > 1}


def junction_positions(strings: List[str], k: int, both: bool) -> List[List[int]]:
    J = junction_kmers(strings, k, both)
    return [[i for i in range(len(s) - k + 1) if s[i:i + k] in J] for s in strings]


def compacted_paths(strings: Iterable[str], k: int, both: bool) -> Set[Tuple[str, ...]]:
    """Maximal non-branching paths, found by walking the explicit graph."""
    strings = list(strings)
    V, E, _ = graph(strings, k, both)
    J = junction_kmers(strings, k, both)
    succ: Dict[str, Set[str]] = defaultdict(set)
    for e in E:
        succ[e[:-1]].add(e[1:])
    paths = set()
    for u in J:
        for w in succ[u]:
            path = [u, w]
            while path[-1] not in J:
                nxt = succ[path[-1]]
                assert len(nxt) == 1, "a non-junction has one successor"
                path.append(next(iter(nxt)))
                assert len(path) <= len(V) + 2, "walk did not reach a junction"
            paths.add(tuple(path))
    return paths


def paths_from_positions(strings: List[str], k: int, positions: List[List[int]]
                         ) -> Set[Tuple[str, ...]]:
    """Paths spelled between consecutive junction positions (Observation 1)."""
    out = set()
    for s, pos in zip(strings, positions):
        pos = sorted(int(p) for p in pos)
        for a, b in zip(pos, pos[1:]):
            out.add(tuple(s[i:i + k] for i in range(a, b + 1)))
    return out
