// Host-side geometry: nozzle voxeliser and the fluid-only sparse index.
//
// Storage layout ("slots"): the active cells of each row (fixed y, z) are
// stored x-contiguously; a row occupies [xb, xe) rounded outward to CHUNK
// boundaries, so slot = row_base[row] + x with row_base a multiple of CHUNK.
// Cells inside a row's span that are solid become padding slots (never
// updated, never pulled from).  Each slot carries a 32-bit link word: one
// bounce-back bit per population, the node type and, for inlet/outlet nodes,
// the direction of the interior partner used by the extrapolation.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "lbm_internal.h"

namespace lbm {

static inline int64_t box_index(int x, int y, int z, int nx, int ny) {
    return (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
}

std::string build_index(const uint8_t *flags, int nx, int ny, int nz, int periodic, HostIndex &out) {
    const int64_t ncell = (int64_t)nx * ny * nz;
    for (int64_t b = 0; b < ncell; ++b)
        if (flags[b] > LBM_OUTLET) {
            char msg[128];
            snprintf(msg, sizeof msg, "flag value %d at cell %lld is not SOLID/FLUID/INLET/OUTLET", (int)flags[b],
                     (long long)b);
            return msg;
        }
    const int64_t nrows = (int64_t)ny * nz;
    if (nrows > INT32_MAX) return "too many rows";
    out = HostIndex();
    out.row_base.assign((size_t)nrows, 0);
    std::vector<int> xb((size_t)nrows, -1), xe((size_t)nrows, -1);
    for (int64_t r = 0; r < nrows; ++r) {
        const uint8_t *row = flags + r * nx;
        for (int x = 0; x < nx; ++x)
            if (row[x] != LBM_SOLID) {
                if (xb[r] < 0) xb[r] = x;
                xe[r] = x + 1;
            }
    }
    int64_t next = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        if (xb[r] < 0) continue;
        const int lo = xb[r] & ~(CHUNK - 1);
        const int hi = (xe[r] + CHUNK - 1) & ~(CHUNK - 1);
        out.row_base[r] = (int32_t)(next - lo);
        for (int x0 = lo; x0 < xe[r]; x0 += CHUNK) out.chunks.push_back(make_int2((int)r, x0));
        next += hi - lo;
        if (next > (int64_t)INT32_MAX - 64) return "lattice too large for 32-bit slot indices";
    }
    out.nslots = (next + 63) & ~(int64_t)63;
    if (out.nslots == 0) return "geometry has no active cells";
    if ((int64_t)out.chunks.size() > (int64_t)INT32_MAX / CHUNK) return "too many chunks";
    out.mask.assign((size_t)out.nslots, (uint32_t)TYPE_PAD << TYPE_SHIFT);

    const bool px = periodic & LBM_PERIODIC_X, py = periodic & LBM_PERIODIC_Y, pz = periodic & LBM_PERIODIC_Z;
    auto flag_at = [&](int x, int y, int z, bool &inside) -> int {
        inside = true;
        if (x < 0 || x >= nx) { if (!px) { inside = false; return LBM_SOLID; } x = (x + nx) % nx; }
        if (y < 0 || y >= ny) { if (!py) { inside = false; return LBM_SOLID; } y = (y + ny) % ny; }
        if (z < 0 || z >= nz) { if (!pz) { inside = false; return LBM_SOLID; } z = (z + nz) % nz; }
        return flags[box_index(x, y, z, nx, ny)];
    };
    static const int dirs[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t b = box_index(x, y, z, nx, ny);
                const int fl = flags[b];
                if (fl == LBM_SOLID) continue;
                const int64_t r = (int64_t)y + (int64_t)ny * z;
                const int32_t slot = out.row_base[r] + x;
                uint32_t m = 0;
                for (int i = 0; i < 27; ++i) {
                    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
                    bool inside;
                    if (flag_at(x - cx, y - cy, z - cz, inside) == LBM_SOLID) m |= 1u << i;
                }
                uint32_t type = TYPE_FLUID, dir = 0;
                if (fl == LBM_INLET || fl == LBM_OUTLET) {
                    type = fl == LBM_INLET ? TYPE_INLET : TYPE_OUTLET;
                    int count = 0;
                    for (int k = 0; k < 6; ++k) {
                        bool inside;
                        if (flag_at(x + dirs[k][0], y + dirs[k][1], z + dirs[k][2], inside) == LBM_FLUID) {
                            ++count;
                            dir = (uint32_t)k;
                        }
                    }
                    if (count != 1) {
                        char msg[160];
                        snprintf(msg, sizeof msg,
                                 "%s node (%d,%d,%d) needs exactly one FLUID axis neighbour, has %d",
                                 fl == LBM_INLET ? "inlet" : "outlet", x, y, z, count);
                        return msg;
                    }
                }
                out.mask[(size_t)slot] = m | (type << TYPE_SHIFT) | (dir << DIR_SHIFT);
                out.slot_of_active.push_back(slot);
                out.box_of_active.push_back(b);
            }
    out.n_active = (int64_t)out.slot_of_active.size();
    return "";
}

}  // namespace lbm

// Nozzle voxeliser (C ABI, declared in lbm.h).
extern "C" lbm_status lbm_make_nozzle(int32_t D, int32_t d, int32_t L_in, int32_t L_cone, int32_t L_throat,
                                      int32_t L_total, double half_angle_deg, uint8_t *out) {
    if (!out || D <= 0 || d <= 0 || d > D || L_in < 0 || L_throat < 0 || L_total <= 0) return LBM_ERR_ARG;
    if (!(half_angle_deg > 0.0 && half_angle_deg < 90.0)) return LBM_ERR_ARG;
    const double slope = std::tan(half_angle_deg * (3.14159265358979323846 / 180.0));
    if (L_cone < 0) L_cone = (int32_t)std::nearbyint((D - d) / 2.0 / slope);  // ties to even
    for (int z = 0; z < L_total; ++z) {
        const double zc = z + 0.5;
        double r;
        if (zc < L_in)
            r = D / 2.0;
        else if (zc < L_in + L_cone)
            r = std::fmax(D / 2.0 - (zc - L_in) * slope, d / 2.0);
        else if (zc < L_in + L_cone + L_throat)
            r = d / 2.0;
        else
            r = D / 2.0;
        for (int y = 0; y < D; ++y)
            for (int x = 0; x < D; ++x) {
                const double rx = x + 0.5 - D / 2.0, ry = y + 0.5 - D / 2.0;
                uint8_t f = (ry * ry + rx * rx <= r * r) ? LBM_FLUID : LBM_SOLID;
                if (f == LBM_FLUID && z == 0) f = LBM_INLET;
                if (f == LBM_FLUID && z == L_total - 1) f = LBM_OUTLET;
                out[((size_t)z * D + y) * D + x] = f;
            }
    }
    return LBM_OK;
}
