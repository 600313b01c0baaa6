"""The paper's damping parameters (oracle copy; test infrastructure only).

Table relaxParam lists the damping w per level for each smoother, found by
trial and error (Section 5.2).  Row 1 is the fine-level relaxation, rows 2-4
the first to third coarse levels.  The paper states that these suffice for up
to 5 levels and that deeper cycles are not sensitive to the extra values; the
levels beyond the table reuse the last row (reading).  Patches with no column
(2D/3D full, 3D RB) use the plus-patch column (reading).
"""
from __future__ import annotations

DAMPING = {
    2: {
        "jacobi": [0.89, 0.9, 0.3, 0.71],
        "element": [0.97, 0.66, 0.48, 0.88],
        "plus": [0.87, 0.57, 0.55, 0.74],
        "rb": [0.83, 0.5, 0.4, 0.65],
    },
    3: {
        "jacobi": [0.6, 0.4, 0.3, 0.5],
        "element": [1.1, 0.7, 0.45, 0.6],
        "plus": [0.92, 0.55, 0.45, 0.55],
    },
}


def damping(dim: int, patch: str, level: int) -> float:
    """Damping of the smoother `patch` on `level` (0 = finest)."""
    table = DAMPING[dim]
    col = table.get(patch, table["plus"])
    return col[min(level, len(col) - 1)]
