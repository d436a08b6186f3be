"""Seeded synthetic inputs: rigid 3-site water boxes, trajectory frames and
parameter sets.

This package generates inputs only. It holds none of the pair-interaction
arithmetic: no cutoff test, no minimum-image pair sum, no force or energy.
Both the CPU oracle (``oracle/``) and the CUDA path read their inputs from
here, so that the two see the same bits.
"""
from .water import (  # noqa: F401
    WaterBox,
    water_box,
    water_box_for_atoms,
    box_edge,
    ewald_beta,
    random_walk_frames,
    diff_params,
    combine_geometric,
    batch_boxes,
    WATER_Q_O,
    WATER_Q_H,
    WATER_C6,
    WATER_C12,
    DENSITY_WATERS_PER_NM3,
)
