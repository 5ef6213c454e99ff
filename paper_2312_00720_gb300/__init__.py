"""GB300 (sm_103a) join and grouped aggregation: radix-partitioned hash join with
GFTR materialization feeding hash-, sort- and partition-based group-bys, behind
the C-ABI declared in include/gj.h."""
