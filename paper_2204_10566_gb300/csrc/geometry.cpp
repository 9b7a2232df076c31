// Host-side geometry: nozzle voxeliser and the fluid-only sparse index.
//
// Storage layout ("slots"): rows are the lines of the box along one axis, the
// row axis (x, or z for lattices longer in z than in x), over the box
// extended by one layer in the two cross axes.  In storage coordinates
// (p along the row axis, a and b across it; (p, a, b) = (x, y, z) for rows
// along x and (z, x, y) for rows along z), row = (a+1) + (n_a+2)(b+1).  A row
// stores, p-contiguously, every position that the step kernel reads or
// writes in it: its active cells, the ghost positions of wall links (a solid
// or outside position p - c_p next to an active fluid cell) and, for a
// periodic row axis, the two wrap-around copies at p = -1 and p = n_p.  Each
// row's stored range is rounded outward to CHUNK boundaries, so
// slot = base(row) + p with base a multiple of CHUNK.  Solid cells inside a
// stored range are padding.
//
// Because every pull source has a slot (an active cell, a ghost slot holding
// the reflected population, or a periodic copy), the kernel's gather is
// branch-free: slot = nb[j] + p - c_p, with nb the row's nine neighbour
// bases, j = (c_a + 1) + 3 (c_b + 1).  Long rows (the flow axis of a nozzle)
// leave few padding lanes and few row ends, where the pulls straddle sectors.
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

int choose_row_axis(int nx, int ny, int nz, int requested) {
    (void)ny;
    if (requested == LBM_ROWS_X) return 0;
    if (requested == LBM_ROWS_Z) return 2;
    return nz > nx ? 2 : 0;  // the longer of x and z
}

namespace {

// Storage coordinates of a lattice whose rows run along axis ax (0: x, 2: z).
struct Frame {
    int ax, nx, ny, nz;
    int np, na, nb;     // extents along the row, and across it
    bool pp, pa, pb;    // periodic along the row, across it
    Frame(int ax_, int nx_, int ny_, int nz_, int periodic) : ax(ax_), nx(nx_), ny(ny_), nz(nz_) {
        const bool px = periodic & LBM_PERIODIC_X, py = periodic & LBM_PERIODIC_Y, pz = periodic & LBM_PERIODIC_Z;
        if (ax == 0) {
            np = nx, na = ny, nb = nz, pp = px, pa = py, pb = pz;
        } else {
            np = nz, na = nx, nb = ny, pp = pz, pa = px, pb = py;
        }
    }
    // box index of storage position (p, a, b), all inside the box
    int64_t box(int p, int a, int b) const {
        return ax == 0 ? box_index(p, a, b, nx, ny) : box_index(a, b, p, nx, ny);
    }
    // storage position of physical cell (x, y, z)
    void from_xyz(int x, int y, int z, int &p, int &a, int &b) const {
        if (ax == 0) {
            p = x, a = y, b = z;
        } else {
            p = z, a = x, b = y;
        }
    }
    // storage components of direction i (physical c = (i%3-1, (i/3)%3-1, i/9-1))
    void dir(int i, int &cp, int &ca, int &cb) const {
        const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
        if (ax == 0) {
            cp = cx, ca = cy, cb = cz;
        } else {
            cp = cz, ca = cx, cb = cy;
        }
    }
};

}  // namespace

std::string build_index(const uint8_t *flags, int nx, int ny, int nz, int periodic, HostIndex &out,
                        int64_t max_slots, int row_axis) {
    const int64_t ncell = (int64_t)nx * ny * nz;
    for (int64_t b = 0; b < ncell; ++b)
        if (flags[b] > LBM_OUTLET) {
            char msg[128];
            snprintf(msg, sizeof msg, "flag value %d at cell %lld is not SOLID/FLUID/INLET/OUTLET", (int)flags[b],
                     (long long)b);
            return msg;
        }
    out = HostIndex();
    const Frame F(choose_row_axis(nx, ny, nz, row_axis), nx, ny, nz, periodic);
    if (F.np > (int)CHUNK_X0_MASK) return "lattice too long along its row axis (at most 2^20 - 1 cells)";
    const int na_e = F.na + 2, nb_e = F.nb + 2;
    const int64_t nrows = (int64_t)na_e * nb_e;
    if (nrows > INT32_MAX / 4) return "too many rows";
    out.row_axis = F.ax;
    out.n_row = F.np;
    out.na_e = na_e;
    out.nb_e = nb_e;
    auto row_of = [&](int a, int b) -> int64_t { return (int64_t)(a + 1) + (int64_t)na_e * (b + 1); };
    // resolve a pull source (p, a, b) (each coordinate at most one step
    // outside the box): returns its flag (SOLID when outside a non-periodic
    // face) and the cross coordinates used for storage (wrapped when
    // periodic; p is wrapped only for the flag lookup).
    auto source = [&](int p, int a, int b, int &as, int &bs) -> int {
        bool outside = false;
        int pw = p, aw = a, bw = b;
        if (p < 0 || p >= F.np) { if (F.pp) pw = (p + F.np) % F.np; else outside = true; }
        if (a < 0 || a >= F.na) { if (F.pa) aw = (a + F.na) % F.na; else outside = true; }
        if (b < 0 || b >= F.nb) { if (F.pb) bw = (b + F.nb) % F.nb; else outside = true; }
        as = F.pa ? aw : a;
        bs = F.pb ? bw : b;
        if (outside) return LBM_SOLID;
        return flags[F.box(pw, aw, bw)];
    };

    std::vector<int> need_lo((size_t)nrows, INT_MAX), need_hi((size_t)nrows, INT_MIN);
    std::vector<int> act_lo((size_t)nrows, INT_MAX), act_hi((size_t)nrows, INT_MIN);  // fluid cells
    auto need = [&](int64_t r, int p) {
        if (p < need_lo[r]) need_lo[r] = p;
        if (p > need_hi[r]) need_hi[r] = p;
    };
    for (int b = 0; b < F.nb; ++b)
        for (int a = 0; a < F.na; ++a)
            for (int p = 0; p < F.np; ++p) {
                const int fl = flags[F.box(p, a, b)];
                if (fl == LBM_SOLID) continue;
                const int64_t r = row_of(a, b);
                need(r, p);
                if (fl == LBM_FLUID) {
                    if (p < act_lo[r]) act_lo[r] = p;
                    if (p > act_hi[r]) act_hi[r] = p;
                }
                if (F.pp && p == F.np - 1) need(r, -1);
                if (F.pp && p == 0) need(r, F.np);
                if (fl != LBM_FLUID) continue;
                for (int i = 0; i < 27; ++i) {
                    int cp, ca, cb, as, bs;
                    F.dir(i, cp, ca, cb);
                    if (source(p - cp, a - ca, b - cb, as, bs) == LBM_SOLID) need(row_of(as, bs), p - cp);
                }
            }
    std::vector<int32_t> base((size_t)nrows, 0);
    // Storage starts n_p + 8 slots in: every chunk lane (fluid or not) then
    // pulls from a non-negative slot, so the 32-bit unsigned element offsets
    // of the step kernel never wrap (a non-fluid lane may pull from before the
    // first stored cell of a neighbour row).
    int64_t next = ((int64_t)F.np + 8 + CHUNK - 1) / CHUNK * CHUNK;
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
    for (int b = 0; b < F.nb; ++b)
        for (int a = 0; a < F.na; ++a) {
            const int64_t r = row_of(a, b);
            if (need_lo[r] == INT_MAX) continue;
            for (int j = 0; j < 9; ++j) {
                const int ca = j % 3 - 1, cb = j / 3 - 1;
                int aa = a - ca, bb = b - cb;
                if (F.pa) aa = (aa + F.na) % F.na;
                if (F.pb) bb = (bb + F.nb) % F.nb;
                out.row_nb[(size_t)r * ROW_RECORD_INTS + j] = base[row_of(aa, bb)];
            }
        }

    // link words, inlet/outlet nodes and the active order (increasing box index)
    static const int dirs[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t bx = box_index(x, y, z, nx, ny);
                const int fl = flags[bx];
                if (fl == LBM_SOLID) continue;
                int p, a, b;
                F.from_xyz(x, y, z, p, a, b);
                const int32_t slot = base[row_of(a, b)] + p;
                uint32_t m = 0, type = TYPE_FLUID, dir = 0;
                if (fl == LBM_FLUID) {
                    for (int i = 0; i < 27; ++i) {
                        int cp, ca, cb, as, bs;
                        F.dir(i, cp, ca, cb);
                        if (source(p - cp, a - ca, b - cb, as, bs) == LBM_SOLID) {
                            m |= 1u << i;
                            ++out.n_ghost;
                        }
                    }
                } else {
                    type = fl == LBM_INLET ? TYPE_INLET : TYPE_OUTLET;
                    int count = 0;
                    for (int k = 0; k < 6; ++k) {
                        int dp, da, db, as, bs;
                        F.from_xyz(dirs[k][0], dirs[k][1], dirs[k][2], dp, da, db);
                        if (source(p + dp, a + da, b + db, as, bs) == LBM_FLUID) {
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
                    out.bnodes.push_back(make_int4(p, (int)row_of(a, b), slot, (int)out.mask[(size_t)slot]));
                out.slot_of_active.push_back(slot);
                out.box_of_active.push_back(bx);
            }
    out.n_active = (int64_t)out.slot_of_active.size();
    if (out.n_active == 0) return "geometry has no active cells";

    // Non-active slots: bit i marks population array i as read there (the
    // ghost slot of a wall link, or a periodic copy along the rows).  The
    // fluid kernel writes every other array of a non-fluid chunk lane with
    // filler, so that the 32-byte sectors at row ends are written whole.
    for (int b = 0; b < F.nb; ++b)
        for (int a = 0; a < F.na; ++a)
            for (int p = 0; p < F.np; ++p) {
                const int fl = flags[F.box(p, a, b)];
                if (fl == LBM_SOLID) continue;
                const int64_t r = row_of(a, b);
                for (int i = 0; i < 27; ++i) {
                    int cp, ca, cb, as, bs;
                    F.dir(i, cp, ca, cb);
                    if (F.pp && p == F.np - 1 && cp == 1) out.mask[(size_t)(base[r] - 1)] |= 1u << i;
                    if (F.pp && p == 0 && cp == -1) out.mask[(size_t)(base[r] + F.np)] |= 1u << i;
                    if (fl == LBM_FLUID && source(p - cp, a - ca, b - cb, as, bs) == LBM_SOLID)
                        out.mask[(size_t)(base[row_of(as, bs)] + p - cp)] |= 1u << i;
                }
            }

    // Chunk records over each row's fluid cells.  A chunk whose eight slots
    // hold no fluid cell and nothing that is read (a solid stretch inside a
    // row's stored range) is left out.
    for (int b = 0; b < F.nb; ++b)
        for (int a = 0; a < F.na; ++a) {
            const int64_t r = row_of(a, b);
            if (act_lo[r] == INT_MAX) continue;
            for (int p0 = (int)std::floor(act_lo[r] / (double)CHUNK) * CHUNK; p0 <= act_hi[r]; p0 += CHUNK) {
                uint32_t lanes = 0, read = 0;
                for (int l = 0; l < CHUNK; ++l) {
                    const int p = p0 + l;
                    if (p < F.np && flags[F.box(p, a, b)] == LBM_FLUID) lanes |= 1u << l;
                    const uint32_t m = out.mask[(size_t)(base[r] + p)];
                    if (((m >> TYPE_SHIFT) & 3u) != TYPE_PAD || (m & LINK_MASK)) read |= 1u << l;
                }
                if (!lanes && !read) continue;
                out.chunks.push_back(make_int2((int)r, (int)((uint32_t)p0 | (lanes << CHUNK_LANES_SHIFT))));
            }
        }
    if ((int64_t)out.chunks.size() > (int64_t)INT32_MAX / CHUNK) return "too many chunks";
    out.tiles = build_tiles(out.chunks, out.row_nb, out.mask, F.np, F.pp);
    out.pair_items = build_pair_items(out.tiles);
    out.rest_chunks = build_rest_chunks(out.chunks, out.tiles, out.pair_items);
    return "";
}

std::vector<int2> build_pair_items(const std::vector<int32_t> &tiles) {
    const int64_t nt = (int64_t)tiles.size() / TILE_INTS;
    auto fast = [&](int64_t t) { return ((uint32_t)tiles[(size_t)t * TILE_INTS] & TILE_FAST) != 0u; };
    std::vector<int2> items;
    for (int64_t t = 0; t + 1 < nt;) {
        if (fast(t) && fast(t + 1)) {
            items.push_back(make_int2((int)t, (int)t + 1));
            t += 2;
        } else {
            t += 1;
        }
    }
    return items;
}

std::vector<int2> build_rest_chunks(const std::vector<int2> &chunks, const std::vector<int32_t> &tiles,
                                    const std::vector<int2> &pairs) {
    const int64_t nt = (int64_t)tiles.size() / TILE_INTS;
    std::vector<uint8_t> paired((size_t)nt, 0);
    for (const int2 &it : pairs) paired[(size_t)it.x] = paired[(size_t)it.y] = 1;
    std::vector<int2> rest;
    size_t c = 0;  // first chunk of tile t: the tiles hold the chunks in order, 8 present lanes each
    for (int64_t t = 0; t < nt; ++t) {
        const size_t n = (size_t)__builtin_popcount((uint32_t)tiles[(size_t)t * TILE_INTS + 2]) / CHUNK;
        if (!paired[(size_t)t]) rest.insert(rest.end(), chunks.begin() + c, chunks.begin() + c + n);
        c += n;
    }
    return rest;
}

std::vector<int32_t> build_tiles(const std::vector<int2> &chunks, const std::vector<int32_t> &row_nb,
                                 const std::vector<uint32_t> &mask, int n_row, bool periodic_row) {
    std::vector<int32_t> tiles;
    int row = -1, p0 = 0, n = 0;  // the open tile
    uint32_t fluid = 0, present = 0;
    auto flush = [&]() {
        if (n == 0) return;
        // fast: 32 fluid cells without wall links, none writing a wrap-around copy
        bool fast = fluid == 0xFFFFFFFFu && !(periodic_row && (p0 == 0 || p0 + 31 >= n_row - 1));
        const int32_t base = row_nb[(size_t)row * ROW_RECORD_INTS + 4];
        for (int l = 0; fast && l < 32; ++l) fast = (mask[(size_t)(base + p0 + l)] & LINK_MASK) == 0u;
        tiles.push_back((int32_t)((uint32_t)p0 | (fast ? TILE_FAST : 0u)));
        tiles.push_back((int32_t)fluid);
        tiles.push_back((int32_t)present);
        for (int j = 0; j < 9; ++j) tiles.push_back(row_nb[(size_t)row * ROW_RECORD_INTS + j]);
        n = 0;
    };
    for (const int2 &c : chunks) {
        const int x0 = (int)((uint32_t)c.y & CHUNK_X0_MASK);
        const uint32_t lanes = ((uint32_t)c.y >> CHUNK_LANES_SHIFT) & 0xFFu;
        if (n == 0 || n == 4 || c.x != row || x0 != p0 + CHUNK * n) {
            flush();
            row = c.x;
            p0 = x0;
            fluid = present = 0;
        }
        fluid |= lanes << (CHUNK * n);
        present |= 0xFFu << (CHUNK * n);
        ++n;
    }
    flush();
    return tiles;
}

// Structural invariants of an index, re-derived independently of how
// build_index produced it: chunk records, alignment and bounds of every
// slot the kernels touch, and the pull slot of every link of every fluid
// cell.  Positions are written in storage coordinates (p along the row
// axis, a and b across it) with their own mapping from the box.
std::string validate_index(const HostIndex &ix, const uint8_t *flags, int nx, int ny, int nz, int periodic) {
    const int64_t ns = ix.nslots;
    const bool zrows = ix.row_axis == 2;
    if (ix.row_axis != 0 && !zrows) return "row axis";
    const int np = zrows ? nz : nx, na = zrows ? nx : ny, nb = zrows ? ny : nz;
    const bool px = periodic & LBM_PERIODIC_X, py = periodic & LBM_PERIODIC_Y, pz = periodic & LBM_PERIODIC_Z;
    const bool pp = zrows ? pz : px, pa = zrows ? px : py, pb = zrows ? py : pz;
    if (ix.n_row != np || ix.na_e != na + 2 || ix.nb_e != nb + 2) return "row grid";
    const int64_t nrows = (int64_t)ix.na_e * ix.nb_e;
    if (ix.row_nb.size() != (size_t)nrows * ROW_RECORD_INTS) return "row record count";
    // box index of storage position (p, a, b) inside the box, and back
    auto box_of = [&](int p, int a, int b) -> int64_t {
        const int x = zrows ? a : p, y = zrows ? b : a, z = zrows ? p : b;
        return (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
    };
    auto pab_of = [&](int64_t bx, int &p, int &a, int &b) {
        const int x = (int)(bx % nx), y = (int)((bx / nx) % ny), z = (int)(bx / ((int64_t)nx * ny));
        p = zrows ? z : x;
        a = zrows ? x : y;
        b = zrows ? y : z;
    };
    std::vector<uint8_t> seen((size_t)nx * ny * nz, 0);

    for (const int2 &c : ix.chunks) {
        const int r = c.x, p0 = (int)((uint32_t)c.y & CHUNK_X0_MASK);
        const uint32_t lanes = ((uint32_t)c.y >> CHUNK_LANES_SHIFT) & 0xFFu;
        if (r < 0 || r >= nrows || p0 % CHUNK) return "bad chunk";
        for (int j = 0; j < 9; ++j)
            if (ix.row_nb[(size_t)r * ROW_RECORD_INTS + j] % CHUNK) return "row base not chunk aligned";
        const int a = r % ix.na_e - 1, b = r / ix.na_e - 1;
        for (int l = 0; l < CHUNK; ++l) {
            if (!((lanes >> l) & 1u)) continue;
            const int p = p0 + l;
            if (p >= np || a < 0 || a >= na || b < 0 || b >= nb) return "chunk lane outside the box";
            const int64_t bx = box_of(p, a, b);
            if (flags[bx] != LBM_FLUID || seen[bx]++) return "chunk lane is not a unique fluid cell";
        }
    }
    // Every position the step reads or writes owns its slot: the active
    // cells, their periodic copies along the rows, and the ghost position of
    // every wall link (p - c_p in the pulled row; rows wrap on periodic cross
    // faces).  Two positions sharing a slot (overlapping row ranges, a missing
    // copy) would overwrite each other.
    std::vector<int32_t> slot_of_box((size_t)nx * ny * nz, -1);
    std::vector<int64_t> owner((size_t)ns, -1);
    const int64_t width = (int64_t)np + 2;  // positions -1 .. np of a row
    auto row_e = [&](int a, int b) -> int64_t { return (int64_t)(a + 1) + (int64_t)ix.na_e * (b + 1); };
    auto claim = [&](int64_t row, int p, int64_t s) -> bool {
        if (s < 0 || s >= ns) return false;
        const int64_t key = row * width + (p + 1);
        int64_t &o = owner[(size_t)s];
        if (o < 0) o = key;
        return o == key;
    };
    for (int64_t k = 0; k < ix.n_active; ++k) {
        const int64_t bx = ix.box_of_active[k];
        int p, a, b;
        pab_of(bx, p, a, b);
        const int32_t *nb_ = &ix.row_nb[(size_t)row_e(a, b) * ROW_RECORD_INTS];
        slot_of_box[(size_t)bx] = ix.slot_of_active[k];
        if (!claim(row_e(a, b), p, ix.slot_of_active[k])) return "two positions share the slot of an active cell";
        if (pp && p == np - 1 && !claim(row_e(a, b), -1, (int64_t)nb_[4] - 1)) return "periodic copy slot";
        if (pp && p == 0 && !claim(row_e(a, b), np, (int64_t)nb_[4] + np)) return "periodic copy slot";
    }
    // pulls of every fluid cell land on stored slots: exactly the slot of an
    // active source inside the box, else a non-active slot of the pulled
    // position that marks the pulled array as read (never filled)
    for (int64_t k = 0; k < ix.n_active; ++k) {
        const int64_t bx = ix.box_of_active[k];
        if (flags[bx] != LBM_FLUID) continue;
        int p, a, b;
        pab_of(bx, p, a, b);
        const int32_t *nb_ = &ix.row_nb[(size_t)row_e(a, b) * ROW_RECORD_INTS];
        if (nb_[4] + p != ix.slot_of_active[k]) return "slot of an active cell";
        for (int i = 0; i < 27; ++i) {
            const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
            const int cp = zrows ? cz : cx, ca = zrows ? cx : cy, cb = zrows ? cy : cz;
            const int64_t s = (int64_t)nb_[(ca + 1) + 3 * (cb + 1)] + p - cp;
            if (s < 0 || s >= ns) return "pull slot outside the buffer";
            const uint32_t m = ix.mask[(size_t)s];
            if (((m >> TYPE_SHIFT) & 3u) == TYPE_PAD && !((m >> i) & 1u)) return "pulled slot not marked as read";
            int ps = p - cp, as = a - ca, bs = b - cb;
            bool outside = false, wrapped_p = false;
            if (ps < 0 || ps >= np) {
                if (pp) { ps = (ps + np) % np; wrapped_p = true; } else outside = true;
            }
            if (as < 0 || as >= na) { if (pa) as = (as + na) % na; else outside = true; }
            if (bs < 0 || bs >= nb) { if (pb) bs = (bs + nb) % nb; else outside = true; }
            if (!outside && !wrapped_p) {
                const int32_t own = slot_of_box[(size_t)box_of(ps, as, bs)];
                if (own >= 0) {
                    if (s != own) return "pull of an active source misses its slot";
                    continue;
                }
            }
            // ghost of a wall link, or a periodic copy: the pulled row (wrapped
            // on periodic cross faces) at p - c_p
            if (!claim(row_e(pa ? as : a - ca, pb ? bs : b - cb), p - cp, s))
                return "two positions share a ghost or copy slot";
        }
    }
    for (int64_t b = 0; b < (int64_t)seen.size(); ++b)
        if ((flags[b] == LBM_FLUID) != (seen[b] == 1)) return "fluid cell not in exactly one chunk lane";
    // every lane of every chunk (fluid or not) loads its 27 pull slots: they
    // must not precede the buffer (the step kernel's 32-bit offsets are
    // unsigned) nor pass the end of its margin
    const int64_t margin = buffer_margin(np);
    for (const int2 &c : ix.chunks) {
        const int32_t *nb_ = &ix.row_nb[(size_t)c.x * ROW_RECORD_INTS];
        const int p0 = (int)((uint32_t)c.y & CHUNK_X0_MASK);
        for (int l = 0; l < CHUNK; ++l)
            for (int i = 0; i < 27; ++i) {
                const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
                const int cp = zrows ? cz : cx, ca = zrows ? cx : cy, cb = zrows ? cy : cz;
                const int64_t s = (int64_t)nb_[(ca + 1) + 3 * (cb + 1)] + p0 + l - cp;
                if (s < 0 || s >= ns + margin) return "chunk lane pull outside the buffer";
            }
        if ((int64_t)nb_[4] + p0 < 0 || (int64_t)nb_[4] + p0 + CHUNK > ns) return "chunk slots outside the buffer";
    }
    for (const int4 &n : ix.bnodes)
        if (n.z < 0 || n.z >= ns || ix.row_nb[(size_t)n.y * ROW_RECORD_INTS + 4] + n.x != n.z) return "boundary node";

    // Tiles of the tile kernel: every fluid cell in exactly one fluid lane, at
    // its own slot, with the bases of its own row; every lane's pulls (p0 - 1
    // .. p0 + 32 of each neighbour row, checked with a margin of 8) and link
    // words inside the buffer and its margins; the fast flag only on tiles of
    // 32 fluid cells without wall links or wrap-around copies.
    const int64_t nt = (int64_t)ix.tiles.size() / TILE_INTS;
    if ((int64_t)ix.tiles.size() != nt * TILE_INTS) return "tile record size";
    std::vector<int64_t> box_of_slot((size_t)ns, -1);
    for (int64_t k = 0; k < ix.n_active; ++k) box_of_slot[(size_t)ix.slot_of_active[k]] = ix.box_of_active[k];
    std::vector<uint8_t> in_tile((size_t)nx * ny * nz, 0);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *rec = &ix.tiles[(size_t)t * TILE_INTS];
        const bool fast = ((uint32_t)rec[0] & TILE_FAST) != 0u;
        const int p0 = (int)((uint32_t)rec[0] & ~TILE_FAST);
        const uint32_t fl = (uint32_t)rec[1], pr = (uint32_t)rec[2];
        const int32_t *tb = rec + 3;
        if (p0 % CHUNK || (fl & ~pr)) return "tile start or lanes";
        if (fast) {
            if (fl != 0xFFFFFFFFu || (pp && (p0 == 0 || p0 + 31 >= np - 1))) return "fast tile lanes";
            for (int l = 0; l < 32; ++l)
                if (ix.mask[(size_t)(tb[4] + p0 + l)] & LINK_MASK) return "fast tile with a wall link";
        }
        for (int j = 0; j < 9; ++j) {
            const int64_t lo = (int64_t)tb[j] + p0 - 8, hi = (int64_t)tb[j] + p0 + 40;
            if (lo < -margin || hi > ns + margin) return "tile window outside the buffer";
        }
        if ((int64_t)tb[4] + p0 < 0 || (int64_t)tb[4] + p0 + 32 > ns + MASK_MARGIN) return "tile link words";
        for (int l = 0; l < 32; ++l) {
            if (!((pr >> l) & 1u)) continue;
            const int64_t s = (int64_t)tb[4] + p0 + l;
            if (s < 0 || s >= ns) return "tile lane outside the buffer";
            if (!((fl >> l) & 1u)) continue;
            const int64_t bx = box_of_slot[(size_t)s];
            if (bx < 0 || flags[bx] != LBM_FLUID || in_tile[(size_t)bx]++) return "tile lane is not a unique fluid cell";
            int p, a, b;
            pab_of(bx, p, a, b);
            if (p != p0 + l) return "tile lane position";
            for (int j = 0; j < 9; ++j)
                if (ix.row_nb[(size_t)row_e(a, b) * ROW_RECORD_INTS + j] != tb[j]) return "tile bases";
        }
    }
    for (int64_t b = 0; b < (int64_t)in_tile.size(); ++b)
        if ((flags[b] == LBM_FLUID) != (in_tile[b] == 1)) return "fluid cell not in exactly one tile lane";
    // FP16S split: pairs of fast tiles, each tile in at most one pair; the
    // chunks of the pairs' tiles (four full chunks from p0, on the tile's own
    // row) and the rest chunks together are the chunk list, as a multiset
    std::vector<uint8_t> in_pair((size_t)nt, 0);
    using ChunkKey = std::pair<int64_t, uint32_t>;  // (row base slot, chunk word)
    std::vector<ChunkKey> split, whole;
    for (const int2 &it : ix.pair_items) {
        if (it.x < 0 || it.x >= nt || it.y < 0 || it.y >= nt || it.x == it.y) return "pair item tile";
        if (in_pair[(size_t)it.x]++ || in_pair[(size_t)it.y]++) return "tile in two pair items";
        for (const int t : {it.x, it.y}) {
            const int32_t *rec = &ix.tiles[(size_t)t * TILE_INTS];
            if (!((uint32_t)rec[0] & TILE_FAST)) return "pair item of a tile that is not fast";
            const uint32_t p0 = (uint32_t)rec[0] & ~TILE_FAST;
            for (uint32_t k = 0; k < 4; ++k)
                split.emplace_back(rec[3 + 4], (p0 + CHUNK * k) | (0xFFu << CHUNK_LANES_SHIFT));
        }
    }
    auto key = [&](const int2 &c) -> ChunkKey {
        return {ix.row_nb[(size_t)c.x * ROW_RECORD_INTS + 4], (uint32_t)c.y};
    };
    for (const int2 &c : ix.rest_chunks) {
        if (c.x < 0 || (int64_t)c.x >= nrows) return "rest chunk row";
        split.push_back(key(c));
    }
    for (const int2 &c : ix.chunks) whole.push_back(key(c));
    std::sort(split.begin(), split.end());
    std::sort(whole.begin(), whole.end());
    if (split != whole) return "pair tiles and rest chunks do not cover the chunks exactly once";

    return "";
}

}  // namespace lbm

// Host-only check of a flag field and its sparse index (C ABI, lbm.h).
extern "C" lbm_status lbm_check_layout(const uint8_t *flags, int32_t nx, int32_t ny, int32_t nz, int32_t periodic,
                                       int32_t row_axis, int64_t out[8]) {
    if (!flags || nx < 1 || ny < 1 || nz < 1 || (periodic & ~7)) return LBM_ERR_ARG;
    if (row_axis != LBM_ROWS_AUTO && row_axis != LBM_ROWS_X && row_axis != LBM_ROWS_Z) return LBM_ERR_ARG;
    lbm::HostIndex ix;
    if (!lbm::build_index(flags, nx, ny, nz, periodic, ix, 0, row_axis).empty()) return LBM_ERR_ARG;
    if (!lbm::validate_index(ix, flags, nx, ny, nz, periodic).empty()) return LBM_ERR_STATE;
    if (out) {
        out[0] = ix.n_active;
        out[1] = ix.nslots;
        out[2] = (int64_t)ix.row_nb.size() / lbm::ROW_RECORD_INTS;
        out[3] = (int64_t)ix.chunks.size();
        out[4] = (int64_t)ix.bnodes.size();
        out[5] = ix.n_ghost;
        out[6] = (int64_t)ix.na_e * ix.nb_e;
        out[7] = ix.row_axis == 2 ? LBM_ROWS_Z : LBM_ROWS_X;
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
