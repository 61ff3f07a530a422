"""Seeded synthetic chart sets (inputs only; no packing arithmetic)."""
from .charts import (ChartSet, Request, batch256, from_polygons, knees, pareto20k,  # noqa: F401
                     plain64, rectangles, serve_stream, stars, stars2k, WORKLOADS)
