// Host-side geometry: nozzle voxeliser and the fluid-only sparse index.
//
// Storage layout ("slots"): rows are the x-lines of the box extended by one
// layer in y and z (row = (y+1) + (ny+2)(z+1)).  A row stores, x-contiguously,
// every position that the step kernel reads or writes in it: its active
// cells, the ghost positions of wall links (a solid or outside position
// x - c_i next to an active fluid cell x) and, for a periodic x axis, the two
// wrap-around copies at x = -1 and x = nx.  Each row's stored range is
// rounded outward to CHUNK boundaries, so slot = base(row) + x with base a
// multiple of CHUNK.  Solid cells inside a stored range are padding.
//
// Because every pull source x - c_i has a slot (an active cell, a ghost slot
// holding the reflected population, or a periodic copy), the kernel's gather
// is branch-free: slot = nb[j] + x - cx, with nb the row's neighbour bases.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "lbm_internal.h"

namespace lbm {

static inline int64_t box_index(int x, int y, int z, int nx, int ny) {
    return (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
}

std::string build_index(const uint8_t *flags, int nx, int ny, int nz, int periodic, HostIndex &out,
                        int64_t max_slots) {
    const int64_t ncell = (int64_t)nx * ny * nz;
    for (int64_t b = 0; b < ncell; ++b)
        if (flags[b] > LBM_OUTLET) {
            char msg[128];
            snprintf(msg, sizeof msg, "flag value %d at cell %lld is not SOLID/FLUID/INLET/OUTLET", (int)flags[b],
                     (long long)b);
            return msg;
        }
    if (nx > (int)CHUNK_X0_MASK) return "nx too large (at most 2^20 - 1)";
    out = HostIndex();
    const bool px = periodic & LBM_PERIODIC_X, py = periodic & LBM_PERIODIC_Y, pz = periodic & LBM_PERIODIC_Z;
    const int ny_e = ny + 2, nz_e = nz + 2;
    const int64_t nrows = (int64_t)ny_e * nz_e;
    if (nrows > INT32_MAX / 4) return "too many rows";
    out.ny_e = ny_e;
    out.nz_e = nz_e;
    auto row_of = [&](int y, int z) -> int64_t { return (int64_t)(y + 1) + (int64_t)ny_e * (z + 1); };
    // resolve a pull source (x, y, z) (each coordinate at most one step outside
    // the box): returns its flag (SOLID when outside a non-periodic face) and
    // the coordinates used for storage (y, z wrapped when periodic; x wrapped
    // only for the flag lookup).
    auto source = [&](int x, int y, int z, int &ys, int &zs) -> int {
        bool outside = false;
        int xw = x, yw = y, zw = z;
        if (x < 0 || x >= nx) { if (px) xw = (x + nx) % nx; else outside = true; }
        if (y < 0 || y >= ny) { if (py) yw = (y + ny) % ny; else outside = true; }
        if (z < 0 || z >= nz) { if (pz) zw = (z + nz) % nz; else outside = true; }
        ys = py ? yw : y;
        zs = pz ? zw : z;
        if (outside) return LBM_SOLID;
        return flags[box_index(xw, yw, zw, nx, ny)];
    };

    std::vector<int> need_lo((size_t)nrows, INT_MAX), need_hi((size_t)nrows, INT_MIN);
    std::vector<int> act_lo((size_t)nrows, INT_MAX), act_hi((size_t)nrows, INT_MIN);  // fluid cells
    auto need = [&](int64_t r, int x) {
        if (x < need_lo[r]) need_lo[r] = x;
        if (x > need_hi[r]) need_hi[r] = x;
    };
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int fl = flags[box_index(x, y, z, nx, ny)];
                if (fl == LBM_SOLID) continue;
                const int64_t r = row_of(y, z);
                need(r, x);
                if (fl == LBM_FLUID) {
                    if (x < act_lo[r]) act_lo[r] = x;
                    if (x > act_hi[r]) act_hi[r] = x;
                }
                if (px && x == nx - 1) need(r, -1);
                if (px && x == 0) need(r, nx);
                if (fl != LBM_FLUID) continue;
                for (int i = 0; i < 27; ++i) {
                    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
                    int ys, zs;
                    if (source(x - cx, y - cy, z - cz, ys, zs) == LBM_SOLID) need(row_of(ys, zs), x - cx);
                }
            }
    std::vector<int32_t> base((size_t)nrows, 0);
    // Storage starts nx + 8 slots in: every chunk lane (fluid or not) then pulls
    // from a non-negative slot, so the 32-bit unsigned element offsets of the
    // step kernel never wrap (a non-fluid lane may pull from before the first
    // stored cell of a neighbour row).
    int64_t next = ((int64_t)nx + 8 + CHUNK - 1) / CHUNK * CHUNK;
    for (int64_t r = 0; r < nrows; ++r) {
        if (need_lo[r] == INT_MAX) continue;
        const int lo = (int)std::floor(need_lo[r] / (double)CHUNK) * CHUNK;
        const int hi = ((need_hi[r] + 1 + CHUNK - 1) / CHUNK) * CHUNK;
        base[r] = (int32_t)(next - lo);
        next += hi - lo;
        if (next > (int64_t)INT32_MAX / 2) return "lattice too large for 32-bit slot indices";
    }
    out.nslots = (next + 63) & ~(int64_t)63;
    if (max_slots > 0 && out.nslots > max_slots) {  // refused before the per-slot arrays are allocated
        char msg[192];
        snprintf(msg, sizeof msg, "lattice needs %lld storage slots, more than the limit of %lld",
                 (long long)out.nslots, (long long)max_slots);
        return msg;
    }
    out.mask.assign((size_t)out.nslots, (uint32_t)TYPE_PAD << TYPE_SHIFT);
    out.row_nb.assign((size_t)nrows * ROW_RECORD_INTS, 0);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            const int64_t r = row_of(y, z);
            if (need_lo[r] == INT_MAX) continue;
            for (int j = 0; j < 9; ++j) {
                const int cy = j % 3 - 1, cz = j / 3 - 1;
                int yy = y - cy, zz = z - cz;
                if (py) yy = (yy + ny) % ny;
                if (pz) zz = (zz + nz) % nz;
                out.row_nb[(size_t)r * ROW_RECORD_INTS + j] = base[row_of(yy, zz)];
            }
            if (act_lo[r] == INT_MAX) continue;
            for (int x0 = (int)std::floor(act_lo[r] / (double)CHUNK) * CHUNK; x0 <= act_hi[r]; x0 += CHUNK) {
                uint32_t lanes = 0;
                for (int l = 0; l < CHUNK; ++l) {
                    const int x = x0 + l;
                    if (x < nx && flags[box_index(x, y, z, nx, ny)] == LBM_FLUID) lanes |= 1u << l;
                }
                out.chunks.push_back(make_int2((int)r, (int)((uint32_t)x0 | (lanes << CHUNK_LANES_SHIFT))));
            }
        }
    if ((int64_t)out.chunks.size() > (int64_t)INT32_MAX / CHUNK) return "too many chunks";

    static const int dirs[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t b = box_index(x, y, z, nx, ny);
                const int fl = flags[b];
                if (fl == LBM_SOLID) continue;
                const int32_t slot = base[row_of(y, z)] + x;
                uint32_t m = 0, type = TYPE_FLUID, dir = 0;
                if (fl == LBM_FLUID) {
                    for (int i = 0; i < 27; ++i) {
                        const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
                        int ys, zs;
                        if (source(x - cx, y - cy, z - cz, ys, zs) == LBM_SOLID) {
                            m |= 1u << i;
                            ++out.n_ghost;
                        }
                    }
                } else {
                    type = fl == LBM_INLET ? TYPE_INLET : TYPE_OUTLET;
                    int count = 0;
                    for (int k = 0; k < 6; ++k) {
                        int ys, zs;
                        if (source(x + dirs[k][0], y + dirs[k][1], z + dirs[k][2], ys, zs) == LBM_FLUID) {
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
                if (type != TYPE_FLUID)
                    out.bnodes.push_back(make_int4(x, (int)row_of(y, z), slot, (int)out.mask[(size_t)slot]));
                out.slot_of_active.push_back(slot);
                out.box_of_active.push_back(b);
            }
    out.n_active = (int64_t)out.slot_of_active.size();
    if (out.n_active == 0) return "geometry has no active cells";

    // Non-active slots: bit i marks population array i as read there (the
    // ghost slot of a wall link, or a periodic-x copy).  The fluid kernel
    // writes every other array of a non-fluid chunk lane with filler, so that
    // the 32-byte sectors at row ends are written whole.
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int fl = flags[box_index(x, y, z, nx, ny)];
                if (fl == LBM_SOLID) continue;
                const int64_t r = row_of(y, z);
                if (px && x == nx - 1)
                    for (int i = 2; i < 27; i += 3) out.mask[(size_t)(base[r] - 1)] |= 1u << i;
                if (px && x == 0)
                    for (int i = 0; i < 27; i += 3) out.mask[(size_t)(base[r] + nx)] |= 1u << i;
                if (fl != LBM_FLUID) continue;
                for (int i = 0; i < 27; ++i) {
                    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
                    int ys, zs;
                    if (source(x - cx, y - cy, z - cz, ys, zs) == LBM_SOLID)
                        out.mask[(size_t)(base[row_of(ys, zs)] + x - cx)] |= 1u << i;
                }
            }
    return "";
}

// Structural invariants of an index, re-derived independently of how
// build_index produced it: segment and chunk records, alignment and bounds of
// every staged copy, and the pull slot of every link of every fluid cell.
std::string validate_index(const HostIndex &ix, const uint8_t *flags, int nx, int ny, int nz, int periodic) {
    const int64_t ns = ix.nslots;
    const int64_t nrows = (int64_t)ix.ny_e * ix.nz_e;
    if (ix.row_nb.size() != (size_t)nrows * ROW_RECORD_INTS) return "row record count";
    std::vector<uint8_t> seen((size_t)nx * ny * nz, 0);

    for (const int2 &c : ix.chunks) {
        const int r = c.x, x0 = (int)((uint32_t)c.y & CHUNK_X0_MASK);
        const uint32_t lanes = ((uint32_t)c.y >> CHUNK_LANES_SHIFT) & 0xFFu;
        if (r < 0 || r >= nrows || x0 % CHUNK) return "bad chunk";
        for (int j = 0; j < 9; ++j)
            if (ix.row_nb[(size_t)r * ROW_RECORD_INTS + j] % CHUNK) return "row base not chunk aligned";
        const int y = r % ix.ny_e - 1, z = r / ix.ny_e - 1;
        for (int l = 0; l < CHUNK; ++l) {
            if (!((lanes >> l) & 1u)) continue;
            const int x = x0 + l;
            if (x >= nx) return "chunk lane outside the box";
            const int64_t bx = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
            if (flags[bx] != LBM_FLUID || seen[bx]++) return "chunk lane is not a unique fluid cell";
        }
    }
    // Every position the step reads or writes owns its slot: the active
    // cells, their periodic-x copies, and the ghost position of every wall
    // link (x - c_i in the pulled row; rows wrap on periodic y / z faces).
    // Two positions sharing a slot (overlapping row ranges, a missing copy)
    // would overwrite each other.
    const bool px = periodic & LBM_PERIODIC_X, py = periodic & LBM_PERIODIC_Y, pz = periodic & LBM_PERIODIC_Z;
    std::vector<int32_t> slot_of_box((size_t)nx * ny * nz, -1);
    std::vector<int64_t> owner((size_t)ns, -1);
    const int64_t width = (int64_t)nx + 2;  // positions -1 .. nx of a row
    auto row_e = [&](int y, int z) -> int64_t { return (int64_t)(y + 1) + (int64_t)ix.ny_e * (z + 1); };
    auto claim = [&](int64_t row, int x, int64_t s) -> bool {
        if (s < 0 || s >= ns) return false;
        const int64_t key = row * width + (x + 1);
        int64_t &o = owner[(size_t)s];
        if (o < 0) o = key;
        return o == key;
    };
    for (int64_t k = 0; k < ix.n_active; ++k) {
        const int64_t bx = ix.box_of_active[k];
        const int x = (int)(bx % nx), y = (int)((bx / nx) % ny), z = (int)(bx / ((int64_t)nx * ny));
        const int32_t *nb = &ix.row_nb[(size_t)row_e(y, z) * ROW_RECORD_INTS];
        slot_of_box[(size_t)bx] = ix.slot_of_active[k];
        if (!claim(row_e(y, z), x, ix.slot_of_active[k])) return "two positions share the slot of an active cell";
        if (px && x == nx - 1 && !claim(row_e(y, z), -1, (int64_t)nb[4] - 1)) return "periodic copy slot";
        if (px && x == 0 && !claim(row_e(y, z), nx, (int64_t)nb[4] + nx)) return "periodic copy slot";
    }
    // pulls of every fluid cell land on stored slots: exactly the slot of an
    // active source inside the box, else a non-active slot of the pulled
    // position that marks the pulled array as read (never filled)
    for (int64_t k = 0; k < ix.n_active; ++k) {
        const int64_t bx = ix.box_of_active[k];
        if (flags[bx] != LBM_FLUID) continue;
        const int x = (int)(bx % nx), y = (int)((bx / nx) % ny), z = (int)(bx / ((int64_t)nx * ny));
        const int32_t *nb = &ix.row_nb[(size_t)row_e(y, z) * ROW_RECORD_INTS];
        if (nb[4] + x != ix.slot_of_active[k]) return "slot of an active cell";
        for (int i = 0; i < 27; ++i) {
            const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
            const int64_t s = (int64_t)nb[i / 3] + x - cx;
            if (s < 0 || s >= ns) return "pull slot outside the buffer";
            const uint32_t m = ix.mask[(size_t)s];
            if (((m >> TYPE_SHIFT) & 3u) == TYPE_PAD && !((m >> i) & 1u)) return "pulled slot not marked as read";
            int xs = x - cx, ys = y - cy, zs = z - cz;
            bool outside = false, wrapped_x = false;
            if (xs < 0 || xs >= nx) {
                if (px) { xs = (xs + nx) % nx; wrapped_x = true; } else outside = true;
            }
            if (ys < 0 || ys >= ny) { if (py) ys = (ys + ny) % ny; else outside = true; }
            if (zs < 0 || zs >= nz) { if (pz) zs = (zs + nz) % nz; else outside = true; }
            if (!outside && !wrapped_x) {
                const int32_t own = slot_of_box[(size_t)(xs + (int64_t)nx * (ys + (int64_t)ny * zs))];
                if (own >= 0) {
                    if (s != own) return "pull of an active source misses its slot";
                    continue;
                }
            }
            // ghost of a wall link, or a periodic-x copy: the pulled row (wrapped
            // on periodic y / z faces) at x - cx
            if (!claim(row_e(py ? ys : y - cy, pz ? zs : z - cz), x - cx, s))
                return "two positions share a ghost or copy slot";
        }
    }
    for (int64_t b = 0; b < (int64_t)seen.size(); ++b)
        if ((flags[b] == LBM_FLUID) != (seen[b] == 1)) return "fluid cell not in exactly one chunk lane";
    // every lane of every chunk (fluid or not) loads its 27 pull slots: they
    // must not precede the buffer (the step kernel's 32-bit offsets are
    // unsigned) nor pass the end of its margin
    const int64_t margin = buffer_margin(nx);
    for (const int2 &c : ix.chunks) {
        const int32_t *nb = &ix.row_nb[(size_t)c.x * ROW_RECORD_INTS];
        const int x0 = (int)((uint32_t)c.y & CHUNK_X0_MASK);
        for (int l = 0; l < CHUNK; ++l)
            for (int i = 0; i < 27; ++i) {
                const int64_t s = (int64_t)nb[i / 3] + x0 + l - (i % 3 - 1);
                if (s < 0 || s >= ns + margin) return "chunk lane pull outside the buffer";
            }
        if ((int64_t)nb[4] + x0 < 0 || (int64_t)nb[4] + x0 + CHUNK > ns) return "chunk slots outside the buffer";
    }
    for (const int4 &n : ix.bnodes)
        if (n.z < 0 || n.z >= ns || ix.row_nb[(size_t)n.y * ROW_RECORD_INTS + 4] + n.x != n.z) return "boundary node";

    return "";
}

}  // namespace lbm

// Host-only check of a flag field and its sparse index (C ABI, lbm.h).
extern "C" lbm_status lbm_check_layout(const uint8_t *flags, int32_t nx, int32_t ny, int32_t nz, int32_t periodic,
                                       int64_t out[8]) {
    if (!flags || nx < 1 || ny < 1 || nz < 1 || (periodic & ~7)) return LBM_ERR_ARG;
    lbm::HostIndex ix;
    if (!lbm::build_index(flags, nx, ny, nz, periodic, ix).empty()) return LBM_ERR_ARG;
    if (!lbm::validate_index(ix, flags, nx, ny, nz, periodic).empty()) return LBM_ERR_STATE;
    if (out) {
        out[0] = ix.n_active;
        out[1] = ix.nslots;
        out[2] = (int64_t)ix.row_nb.size() / lbm::ROW_RECORD_INTS;
        out[3] = (int64_t)ix.chunks.size();
        out[4] = (int64_t)ix.bnodes.size();
        out[5] = ix.n_ghost;
        out[6] = (int64_t)ix.ny_e * ix.nz_e;
        out[7] = 0;
    }
    return LBM_OK;
}

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
