// Host-side table builders (double precision, no fused multiply-adds).
#pragma once

#include <stdint.h>

#include <vector>

#include "bf_internal.h"

namespace bfi {

struct GeomHost {
    int ne = 0;
    std::vector<double> xe;  // element x positions (m)
    double fnum = 1.0;
    int nx = 1, nz = 1;
    double x0 = 0, x1 = 0, z0 = 0, z1 = 0;
    double fs = 0, f0 = 0, c = 0;
};

// Angle-independent tables of a handle.
struct GeometryHost {
    std::vector<int> ap_first;     // [nx][ne] first row inside the aperture (nz: never)
    std::vector<uint16_t> apcnt;   // [nx][nz] channels inside the aperture
    std::vector<float> rowZ;
    std::vector<float> dx2;        // [ne][nxp] (kappa (x_p - x_i))^2, columns padded
};

// Tables of one angle set and sample count.
struct PlanHost {
    std::vector<int> colK, rowK;
    std::vector<float> colF, rowF;
    std::vector<int> valid;        // [na][ne][nxp][2] first / last counted row (padding: none)
    int wmax = 0, box = 0, group = 1, nsp = 0, rows = 8, align = 2;
};

struct EnvHost {
    int nz = 0, fft_m = 0, bluestein = 0;
    std::vector<float> tw, chirp, bhat;  // interleaved re / im
};

double grid_coord(double lo, double hi, int n, int j);
void geometry_tables(const GeomHost &g, GeometryHost &out);
// rows: rows per thread of the beamforming tile (tile height kWarps * rows);
// stage_bytes: target bytes of sample windows per pipeline stage (sets the
// channels per stage)
void angle_tables(const GeomHost &g, const GeometryHost &geo, int ns,
                  const std::vector<double> &angles, int prec, int rows, int stage_bytes,
                  PlanHost &out);
void bandpass_bins(int nz, double z0, double z1, double c, double f0, int &lo, int &hi);
// Plane-wave f-k mapping of every (angle, Kz bin q = 1 .. nt/2, Kx bin m):
// i0 [na][nt/2][nk] the temporal bin below the mapped position (-1: nothing
// taken), aw [na][nt/2][nk][2] its interpolation weight toward i0 + 1 and the
// spectral weight.  sc: sin, cos of each angle.  stolt: Stolt's mapping of the
// exploding-reflector fit instead of the exact plane-wave mapping.  Double
// precision, evaluated in the order the definitions are written.
void fk_mapping_tables(int ne, int nt, int nk, double pitch, double dz,
                       const std::vector<double> &sc, bool stolt, std::vector<int> &i0,
                       std::vector<float> &aw);
void envelope_tables(int nz, EnvHost &out);

}  // namespace bfi
