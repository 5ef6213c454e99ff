"""The paper's cost models, written out as stated -- TEST INFRASTRUCTURE ONLY.

All costs are in seconds for a global-memory bandwidth ``bg`` in bytes/s; the
paper's A100 uses bg = 1555e9 (Sec. 5).

M1 (Sec. 4.1.1): random-access bandwidth B_R ~ B_G / 24, from the 8.52x gap
between unclustered and clustered gathers of 2^27 4-byte items (Table
gather-profile).

M2 (Sec. 4.1.3, SGB GFTR vs GFUR, 4-byte keys and payloads, N tuples, g groups):
    C_S = 68 N / B_G                       -- sort one payload with the key
    C_P = (4 min(24, g) + 8) N / B_G       -- unclustered gather of one payload

M3 (Sec. 4.1.4, PHJ GFTR vs GFUR for one column of a relation of N tuples with
M = mr N matches, 16 radix bits):
    C_1 = 104 M / B_G                      -- unclustered gather
    C_2 = (36 N + 12 M) / B_G              -- partition then clustered gather

M4 (Sec. 4.4, dictionary encoding for SGB, k-byte keys, p payload columns):
    C_1 = p (k N + 2 k N (k + 4)) / B_G
    C_2 = D(N, g) + p (4 N + ceil(log2(g) / 8) 16 N) / B_G
    D(N, g) = k g / B_G + (k+4) g / (B_M / min(g, 24))
            + (k N + 4 N) / B_G + (k+4) N / (B_M / min(g, 24))
  where B_M is the bandwidth of the memory level the non-empty hash entries
  fit in. The paper gives B_L1 ~ 12 B_G and B_L2 ~ 4.5 B_G for the A100 but not
  the capacities; reading taken here: (k+4) g bytes <= 192 KB -> L1, <= 40 MB ->
  L2, else global memory (the A100's L1 and L2 sizes from Sec. 5).
"""
from __future__ import annotations

import math

A100_BG = 1555e9
A100_L1_BYTES = 192 * 1024
A100_L2_BYTES = 40 * 1024 * 1024


def random_access_bw(bg: float) -> float:
    """M1: B_R = B_G / 24 (Sec. 4.1.1)."""
    return bg / 24.0


def m2_sort_cost(n: float, bg: float) -> float:
    """C_S: histogram plus four 8-bit passes reading and writing key and payload, 17 x 4N bytes."""
    return 17.0 * 4.0 * n / bg


def m2_gather_cost(n: float, g: float, bg: float) -> float:
    """C_P: ids and results sequential (8N bytes) + payload read at B_G / min(24, g)."""
    u = min(24.0, g)
    return 2.0 * n * 4.0 / bg + n * 4.0 / max(bg / u, bg / 24.0)


def m2_gftr_wins(g: float) -> bool:
    """SGB-TR beats SGB-UR for one payload column when C_P > C_S, i.e. g >= 16."""
    return m2_gather_cost(1.0, g, 1.0) > m2_sort_cost(1.0, 1.0)


def fig_sgb_model1_estimate_ms(g: float, n: float = 2.0**28, bg: float = A100_BG, ncols: int = 2) -> float:
    """Time(SGB-UR) - Time(SGB-TR) for ncols payload columns: GFUR gathers every
    column (ncols C_P); GFTR sorts every column but the first rides with the key
    as the tuple ids do in GFUR, so it pays (ncols - 1) C_S extra."""
    return (ncols * m2_gather_cost(n, g, bg) - (ncols - 1) * m2_sort_cost(n, bg)) * 1e3


def m3_gfur_cost(m: float, bg: float) -> float:
    """C_1 = read ids + write output (8M) + read input at B_G/24 (4M x 24) = 104 M / B_G."""
    return 2.0 * 4.0 * m / bg + 4.0 * m / random_access_bw(bg)


def m3_gftr_cost(n: float, m: float, bg: float) -> float:
    """C_2 = histogram (4N) + two passes that each read and write key and column (2 x 4 x 4N = 32N)
    + clustered gather of M items reading ids, input and writing output (12 M)."""
    return (4.0 * n + 2.0 * 4.0 * 4.0 * n) / bg + 3.0 * 4.0 * m / bg


def m3_threshold_mr(ncols: int) -> float:
    """Smallest match ratio for which GFTR is cheaper, with the first column riding free."""
    # ncols * C_1(mr N) > (ncols - 1) * (36 N) + ncols * 12 mr N  (per N, per B_G)
    if ncols <= 0:
        return math.inf
    free = 1 if ncols > 1 else 0
    return (ncols - free) * 36.0 / (ncols * (104.0 - 12.0))


def fig_phj_mr_estimate_ms(mr: float, n: float = 2.0**27, bg: float = A100_BG, ncols: int = 2,
                           nrel: int = 2) -> float:
    """Time(PHJ-UR) - Time(PHJ-TR) for nrel relations of n tuples with ncols payloads each;
    GFTR's first payload rides with the key for free (Sec. 4.1.4, last paragraph)."""
    m = mr * n
    per_rel = ncols * m3_gfur_cost(m, bg) - ((ncols - 1) * (4.0 * n + 32.0 * n) / bg + ncols * 12.0 * m / bg)
    return nrel * per_rel * 1e3


def m4_memory_bw(k: int, g: float, bg: float, l1_bytes: float = A100_L1_BYTES,
                 l2_bytes: float = A100_L2_BYTES) -> float:
    """B_M: 12 B_G if the (k+4) g bytes of hash entries fit in L1, 4.5 B_G if in L2, else B_G."""
    entry_bytes = (k + 4) * g
    if entry_bytes <= l1_bytes:
        return 12.0 * bg
    if entry_bytes <= l2_bytes:
        return 4.5 * bg
    return bg


def m4_dictionary_cost(n: float, g: float, k: int, bg: float, bm: float | None = None) -> float:
    """D(N, g): build (k g sequential + (k+4) g random) and probe (k N + 4 N sequential + (k+4) N random)."""
    if bm is None:
        bm = m4_memory_bw(k, g, bg)
    rnd = bm / min(g, 24.0)
    build = k * g / bg + (k + 4) * g / rnd
    probe = (k * n + 4 * n) / bg + (k + 4) * n / rnd
    return build + probe


def m4_passes(g: float) -> int:
    """ceil(log2(g) / 8) radix passes for dictionary codes in {0..g-1}."""
    if g <= 1:
        return 0
    return int(math.ceil(math.log2(g) / 8.0))


def m4_c1(n: float, k: int, p: int, bg: float) -> float:
    """Sort p payload columns with k-byte keys in k 8-bit passes."""
    return p * (k * n + k * n * 2 * (k + 4)) / bg


def m4_c2(n: float, g: float, k: int, p: int, bg: float) -> float:
    """Encode keys, then sort p payload columns on the codes' log2(g) bits."""
    return m4_dictionary_cost(n, g, k, bg) + p * (4 * n + m4_passes(g) * n * 2 * (4 + 4)) / bg


def fig_sgb_model2_estimate_ms(g: float, k: int, n: float = 2.0**28, bg: float = A100_BG, p: int = 1) -> float:
    """Time(SGB-TR) - Time(SGB-DE-TR) = C_1 - C_2 (Fig. sgb-model2)."""
    return (m4_c1(n, k, p, bg) - m4_c2(n, g, k, p, bg)) * 1e3


def m4_min_payloads(g: float, k: int, n: float = 2.0**28, bg: float = A100_BG, pmax: int = 64) -> int | None:
    """Smallest p with C_2 < C_1 (Table de-opt), or None if none up to pmax."""
    for p in range(1, pmax + 1):
        if m4_c2(n, g, k, p, bg) < m4_c1(n, k, p, bg):
            return p
    return None
