// Host-side construction of the transport tables (FP64, rounded to FP32 on
// upload) and of the aperture classification raster.
//
// Stopping power: Bethe-Bloch mass electronic stopping power without shell or
// density-effect corrections and with the full maximum energy transfer.
// Residual range R(E_k) on the 0.1 MeV grid: integral of 1/S from the 0.5 MeV
// transport cut-off, composite Simpson on a 0.001 MeV sub-grid.  E(R) on a
// uniform grid of 4096 residual ranges: inverse of the piecewise-linear R(E).
// Units: R in mm * g/cc (areal range in g/cm^2 times 10).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "tables.h"

namespace vpmc {
namespace {

struct MaterialData {
    double z_over_a, mean_excitation_mev, density, radiation_length_gcm2;
};

// water (patient media, scaled by SPR), PMMA (range shifter), brass 63/37 Cu/Zn
constexpr MaterialData kMaterials[kNMat] = {
    {0.555087, 75.0e-6, 1.00, 36.08},
    {0.539369, 74.0e-6, 1.19, 40.55},
    {0.4573, 330.0e-6, 8.53, 12.9},
};

constexpr double kKBethe = 0.307075;      // MeV cm^2 / mol
constexpr double kElectronMass = 0.51099895;
constexpr double kProtonMass = 938.272;
constexpr double kCutoff = 0.5;

double bethe_mass_stopping_power(const MaterialData& m, double kinetic)
{
    const double gamma = 1.0 + kinetic / kProtonMass;
    const double beta_sq = 1.0 - 1.0 / (gamma * gamma);
    const double bg_sq = beta_sq * gamma * gamma;
    const double mass_ratio = kElectronMass / kProtonMass;
    const double t_max = 2.0 * kElectronMass * bg_sq / (1.0 + 2.0 * gamma * mass_ratio + mass_ratio * mass_ratio);
    const double log_arg = 2.0 * kElectronMass * bg_sq * t_max /
                           (m.mean_excitation_mev * m.mean_excitation_mev);
    return kKBethe * m.z_over_a / beta_sq * (0.5 * std::log(log_arg) - beta_sq);
}

// integral of 10 / S over [a, b] by composite Simpson with `panels` (even) panels
double range_increment(const MaterialData& m, double a, double b, int panels)
{
    const double h = (b - a) / panels;
    double acc = 10.0 / bethe_mass_stopping_power(m, a) + 10.0 / bethe_mass_stopping_power(m, b);
    for (int i = 1; i < panels; ++i) {
        const double w = (i % 2 == 1) ? 4.0 : 2.0;
        acc += w * 10.0 / bethe_mass_stopping_power(m, a + i * h);
    }
    return acc * h / 3.0;
}

void build_material(const MaterialData& m, std::vector<double>& range, std::vector<double>& energy, double& d_range)
{
    range.assign(kNE, 0.0);
    for (int k = 1; k < kNE; ++k) {
        const double upper = 0.1 * k;
        if (upper <= kCutoff) continue;                 // zero range below the cut-off
        const double lower = std::max(0.1 * (k - 1), kCutoff);
        range[k] = range[k - 1] + range_increment(m, lower, upper, 100);
    }
    energy.assign(kNR, 0.0);
    d_range = range[kNE - 1] / (kNR - 1);
    int k = 0;
    for (int j = 0; j < kNR; ++j) {
        if (j == kNR - 1) { energy[j] = 0.1 * (kNE - 1); break; }
        const double r = j * d_range;
        if (r <= 0.0) { energy[j] = kCutoff; continue; }
        while (k + 1 < kNE - 1 && range[k + 1] < r) ++k;
        const double e_lo = std::max(0.1 * k, kCutoff);
        const double e_hi = 0.1 * (k + 1);
        energy[j] = e_lo + (r - range[k]) / (range[k + 1] - range[k]) * (e_hi - e_lo);
    }
}

void curve_props(const double* c15, double hu, double* rho, double* spr)
{
    const double* knot = c15;
    const double* dens = c15 + 5;
    const double* ratio = c15 + 10;
    const double h = std::min(std::max(hu, knot[0]), 3071.0);
    int seg = 0;
    while (seg < 3 && h >= knot[seg + 1]) ++seg;
    const double t = (h - knot[seg]) / (knot[seg + 1] - knot[seg]);
    *rho = dens[seg] + t * (dens[seg + 1] - dens[seg]);
    *spr = ratio[seg] + t * (ratio[seg + 1] - ratio[seg]);
}

bool segment_hits_box(double ax, double ay, double bx, double by, double x0, double y0, double x1, double y1)
{
    // Liang-Barsky clip of segment a->b against the box [x0,x1] x [y0,y1]
    double t0 = 0.0, t1 = 1.0;
    const double dx = bx - ax, dy = by - ay;
    const double p[4] = {-dx, dx, -dy, dy};
    const double q[4] = {ax - x0, x1 - ax, ay - y0, y1 - ay};
    for (int i = 0; i < 4; ++i) {
        if (p[i] == 0.0) {
            if (q[i] < 0.0) return false;
        } else {
            const double t = q[i] / p[i];
            if (p[i] < 0.0) t0 = std::max(t0, t);
            else t1 = std::min(t1, t);
            if (t0 > t1) return false;
        }
    }
    return true;
}

double point_rect_distance(double x, double y, double x0, double y0, double x1, double y1)
{
    const double dx = std::max(std::max(x0 - x, 0.0), x - x1);
    const double dy = std::max(std::max(y0 - y, 0.0), y - y1);
    return std::sqrt(dx * dx + dy * dy);
}

double point_segment_distance(double x, double y, double ax, double ay, double bx, double by)
{
    const double ex = bx - ax, ey = by - ay;
    const double l2 = ex * ex + ey * ey;
    double t = l2 > 0.0 ? ((x - ax) * ex + (y - ay) * ey) / l2 : 0.0;
    t = std::min(std::max(t, 0.0), 1.0);
    const double dx = ax + t * ex - x, dy = ay + t * ey - y;
    return std::sqrt(dx * dx + dy * dy);
}

// Distance between a segment and a rectangle that it does not intersect.
double segment_rect_distance(double ax, double ay, double bx, double by, double x0, double y0, double x1, double y1)
{
    double d = std::min(point_rect_distance(ax, ay, x0, y0, x1, y1), point_rect_distance(bx, by, x0, y0, x1, y1));
    const double cx[4] = {x0, x1, x1, x0}, cy[4] = {y0, y0, y1, y1};
    for (int k = 0; k < 4; ++k) d = std::min(d, point_segment_distance(cx[k], cy[k], ax, ay, bx, by));
    return d;
}

bool crossing_number_inside(const double* xy, int n, double x, double y)
{
    bool inside = false;
    for (int i = 0, j = n - 1; i < n; j = i++) {
        const double xi = xy[2 * i], yi = xy[2 * i + 1], xj = xy[2 * j], yj = xy[2 * j + 1];
        if ((yi > y) != (yj > y) && x < xi + (y - yi) * (xj - xi) / (yj - yi)) inside = !inside;
    }
    return inside;
}

}  // namespace

double pmma_stopping_power_ratio(double kinetic)
{
    return bethe_mass_stopping_power(kMaterials[kPMMA], kinetic) * kMaterials[kPMMA].density /
           bethe_mass_stopping_power(kMaterials[kWater], kinetic);
}

void build_tables(const double* curve15, TablesImage* img)
{
    std::memset(img, 0, sizeof(TablesImage));
    for (int mat = 0; mat < kNMat; ++mat) {
        std::vector<double> range, energy;
        double d_range = 0.0;
        build_material(kMaterials[mat], range, energy, d_range);
        // FP32 values and the FP32 differences to the next entry (zero after
        // the last), as the kernels interpolate them
        for (int k = 0; k < kNEPad; ++k) {
            const float v = (float)range[std::min(k, kNE - 1)];
            const float next = (float)range[std::min(k + 1, kNE - 1)];
            img->R[mat][k] = make_float2(v, next - v);
        }
        for (int j = 0; j < kNR; ++j) {
            const float v = (float)energy[j];
            const float next = (float)energy[std::min(j + 1, kNR - 1)];
            img->Einv[mat][j] = make_float2(v, next - v);
        }
        img->mat[mat].za = (float)kMaterials[mat].z_over_a;
        img->mat[mat].rho = (float)kMaterials[mat].density;
        img->mat[mat].inv_x0 = (float)(1.0 / (kMaterials[mat].radiation_length_gcm2 * 10.0));
        img->mat[mat].inv_dR = (float)(1.0 / d_range);
    }
    for (int i = 0; i < kNHU; ++i) {
        double rho, spr;
        curve_props(curve15, (double)(kHULo + i), &rho, &spr);
        img->hu[i] = make_float2((float)rho, (float)spr);
    }
}

void build_raster(const double* xy, int n, double margin, unsigned char* cells, float* lower, float lo[2], float inv[2],
                  float* diag)
{
    double xmin = xy[0], xmax = xy[0], ymin = xy[1], ymax = xy[1];
    for (int i = 1; i < n; ++i) {
        xmin = std::min(xmin, xy[2 * i]); xmax = std::max(xmax, xy[2 * i]);
        ymin = std::min(ymin, xy[2 * i + 1]); ymax = std::max(ymax, xy[2 * i + 1]);
    }
    // cover the polygon with a margin so that every point outside the raster is
    // outside the polygon and farther than `margin` from its boundary
    const double pad = std::max(0.02 * std::max(xmax - xmin, ymax - ymin) + 0.1, margin);
    xmin -= pad; xmax += pad; ymin -= pad; ymax += pad;
    const double cw = (xmax - xmin) / kRaster, ch = (ymax - ymin) / kRaster;
    lo[0] = (float)xmin; lo[1] = (float)ymin;
    inv[0] = (float)(1.0 / cw); inv[1] = (float)(1.0 / ch);
    *diag = (float)(std::sqrt(cw * cw + ch * ch) * (1.0 + 1e-6) + 1e-4);
    // FP32 placement of a point can move it by a few ulps across a cell border,
    // so a cell is classified only if no edge comes within eps of it
    const double eps = 1e-3 * std::max(cw, ch) + 1e-4 * (std::fabs(xmin) + std::fabs(ymin) + 1.0);
    // rows are independent: split them over the host's threads
    auto rows = [&](int cy_begin, int cy_end) {
    for (int cy = cy_begin; cy < cy_end; ++cy)
        for (int cx = 0; cx < kRaster; ++cx) {
            const double x0 = xmin + cx * cw - eps, x1 = xmin + (cx + 1) * cw + eps;
            const double y0 = ymin + cy * ch - eps, y1 = ymin + (cy + 1) * ch + eps;
            bool edge = false;
            for (int i = 0; i < n && !edge; ++i) {
                const int j = (i + 1) % n;
                edge = segment_hits_box(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], x0, y0, x1, y1);
            }
            unsigned char c = 2;
            if (!edge) c = crossing_number_inside(xy, n, xmin + (cx + 0.5) * cw, ymin + (cy + 0.5) * ch) ? 1 : 0;
            cells[cy * kRaster + cx] = c;
            // lower bound of the distance from any point of the cell to the boundary
            double lb = 0.0;
            if (!edge) {
                lb = 1e300;
                const double rx0 = xmin + cx * cw, rx1 = rx0 + cw, ry0 = ymin + cy * ch, ry1 = ry0 + ch;
                for (int i = 0; i < n; ++i) {
                    const int j = (i + 1) % n;
                    lb = std::min(lb, segment_rect_distance(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1],
                                                            rx0, ry0, rx1, ry1));
                }
                lb = std::max(lb - 1e-4, 0.0);     // margin for the FP32 use of the bound
            }
            lower[cy * kRaster + cx] = (float)lb;
        }
    };
    const int nt = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(rows, t * kRaster / nt, (t + 1) * kRaster / nt);
    rows(0, kRaster / nt);
    for (std::thread& th : pool) th.join();
}

void hu_curve_props(const double* curve15, double hu, double* rho, double* spr) { curve_props(curve15, hu, rho, spr); }

void polygon_curvature(const double* xy, int n, float* kappa)
{
    double twice_area = 0.0;
    for (int i = 0; i < n; ++i) {
        const int j = (i + 1) % n;
        twice_area += xy[2 * i] * xy[2 * j + 1] - xy[2 * j] * xy[2 * i + 1];
    }
    const double orient = twice_area < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) {
        const int a = (i + n - 1) % n, b = (i + 1) % n;
        const double ax = xy[2 * i] - xy[2 * a], ay = xy[2 * i + 1] - xy[2 * a + 1];
        const double bx = xy[2 * b] - xy[2 * i], by = xy[2 * b + 1] - xy[2 * i + 1];
        const double turn = std::atan2(ax * by - ay * bx, ax * bx + ay * by);
        const double half = 0.5 * (std::hypot(ax, ay) + std::hypot(bx, by));
        kappa[i] = (float)(orient * turn / half);
    }
}

}  // namespace vpmc
