"""Seeded synthetic chart sets (inputs only; no packing arithmetic)."""
from .charts import (ChartSet, Request, batch256, batch256_specs, from_polygons, knees,  # noqa: F401
                     pareto20k, plain64, rectangles, serve_specs, serve_stream, stars, stars2k, stars_fast,
                     stars_many, WORKLOADS)
from .fixtures import Stream, serve_stream_fixtures  # noqa: F401
