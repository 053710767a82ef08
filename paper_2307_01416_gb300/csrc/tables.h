// Host-side table and raster builders.
#pragma once

#include "vpmc_internal.cuh"

namespace vpmc {

// curve15 = {hu[5], density[5], spr[5]}
void build_tables(const double* curve15, TablesImage* img);
double pmma_stopping_power_ratio(double kinetic_mev);
void build_raster(const double* xy, int n, unsigned char* cells, float lo[2], float inv[2]);
void hu_curve_props(const double* curve15, double hu, double* rho, double* spr);

}  // namespace vpmc
