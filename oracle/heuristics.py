"""The paper's variant-choice rules -- TEST INFRASTRUCTURE ONLY.

Join (Sec. 5.1.10, the join summary, and Sec. 7): the GFTR partitioned hash join is preferred when
the match ratio is at least 25 %, when the foreign keys are skewed, or when keys
are 8 bytes; otherwise the GFUR partitioned hash join.

Group-by (Fig. groupby-dt): if a sort is mandated, SGB-DE-TR when Table de-opt's
condition holds else SGB-TR; otherwise HGB when its aggregates fit in shared
memory; otherwise SGB (high skew, z >= 1) or PGB-TR.
"""
from __future__ import annotations

from . import cost_models

JOIN_PHJ_TR, JOIN_PHJ_UR, JOIN_NPHJ = "PHJ_TR", "PHJ_UR", "NPHJ"
GB_HGB, GB_SGB, GB_PGB, GB_SGB_DE = "HGB", "SGB", "PGB", "SGB_DE"


def choose_join(mr: float, zipf_theta: float, key_bytes: int, skew_theta: float = 0.5) -> str:
    """Sec. 7: PHJ-TR if mr >= 25 %, skewed FKs or 8-byte keys, else PHJ-UR.

    "Skewed" is read as a Zipf factor of at least ``skew_theta``; the paper's
    skew experiment (Sec. 5.1.7) varies theta but names no threshold."""
    if mr >= 0.25 or zipf_theta >= skew_theta or key_bytes == 8:
        return JOIN_PHJ_TR
    return JOIN_PHJ_UR


def choose_groupby(g_est: float, agg_bytes_per_group: int, smem_bytes: int, zipf_theta: float,
                   key_bytes: int, must_sort: bool = False, n: float = 2.0**28, npayload: int = 1,
                   have_dictionary: bool = False) -> str:
    """Fig. groupby-dt with the group count estimate g_est standing in for g."""
    def sort_branch():
        if have_dictionary:
            p = cost_models.m4_min_payloads(max(g_est, 1.0), key_bytes, n=n)
            if p is not None and npayload >= p:
                return GB_SGB_DE
        return GB_SGB

    if must_sort:
        return sort_branch()
    if g_est * agg_bytes_per_group <= smem_bytes:
        return GB_HGB
    if zipf_theta >= 1.0:
        return sort_branch()
    return GB_PGB
