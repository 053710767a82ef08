// Host-side table and raster builders.
#pragma once

#include "vpmc_internal.cuh"

namespace vpmc {

// curve15 = {hu[5], density[5], spr[5]}
void build_tables(const double* curve15, TablesImage* img);
double pmma_stopping_power_ratio(double kinetic_mev);
// cells: 0 outside, 1 inside, 2 near an edge; lower: per cell a lower bound of
// the distance to the boundary; diag: cell diagonal (plus a margin).  Points
// outside the raster are at least `margin` from the boundary.
void build_raster(const double* xy, int n, double margin, unsigned char* cells, float* lower, float lo[2], float inv[2],
                  float* diag);
// Signed curvature (1/mm) of each polygon vertex: the turning angle at the
// vertex over half the sum of its two edges, positive where the region inside
// the polygon is locally convex (either vertex order).
void polygon_curvature(const double* xy, int n, float* kappa);
void hu_curve_props(const double* curve15, double hu, double* rho, double* spr);

}  // namespace vpmc
