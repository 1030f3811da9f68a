// Host-side check of the tiled gathers' box arithmetic (test infrastructure;
// built and run by tests/test_tile_box_cpu.py, no GPU needed).
//
// For one tile of arrival points and a displacement pattern it runs the same
// __host__ __device__ code the kernels run: bounds_add per point, then
// box_geometry for the tile, then tile_offset per point.  Every tile that the
// geometry marks as fitting must hold every stencil node of every point
// inside the shared-memory box; a tile with a non-finite displacement or one
// of 2^20 cells or more must be marked as not fitting (global-memory path).
// Tile-bounds tables: a box built from the bounds of one displacement field
// (as the backtrace writes them) and used with another, or built from
// arbitrary integers, must never let a point pass in_box with a stencil
// node outside the box; with the field the table was made from, every
// point of a fitting tile must pass.
// Exit status 0 and "OK" on stdout when every case passes.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <limits>
#include <random>

#include "sl_tiled.cuh"

using namespace claire;

namespace {

Grid make_grid(int n1, int n2, int n3)
{
    Grid g;
    g.n1 = n1; g.n2 = n2; g.n3 = n3;
    g.n23 = n2 * n3;
    g.N = static_cast<uint32_t>(n1) * n2 * n3;
    g.h1 = 2.0f * 3.14159265f / n1; g.h2 = 2.0f * 3.14159265f / n2; g.h3 = 2.0f * 3.14159265f / n3;
    g.ih1 = 1.0f / g.h1; g.ih2 = 1.0f / g.h2; g.ih3 = 1.0f / g.h3;
    return g;
}

using Disp = std::function<void(int, int, int, float&, float&, float&)>;

enum Outcome { FITS, GLOBAL, BROKEN };

int g_failures = 0;

// One tile at block (bx, by, bz) of the tiled launch grid.
template <int ORDER, int ES>
Outcome run_tile(const Grid& g, int bx, int by, int bz, const Disp& disp, bool* had_bad)
{
    constexpr int M = Scheme<ORDER>::M;
    constexpr int OFF = Scheme<ORDER>::OFF;
    int lo1 = INT_MAX, lo2 = INT_MAX, lo3 = INT_MAX, hi1 = INT_MIN, hi2 = INT_MIN, hi3 = INT_MIN;
    bool bad = false;
    for (int w = 0; w < TILE2; ++w)
        for (int l = 0; l < TILE3; ++l)
            for (int q = 0; q < TILE1; ++q) {
                const int i = bz * TILE1 + q, j = by * TILE2 + w, k = bx * TILE3 + l;
                if (i >= g.n1 || j >= g.n2 || k >= g.n3) continue;
                float d1, d2, d3;
                disp(i, j, k, d1, d2, d3);
                bounds_add(i, d1, lo1, hi1, bad);
                bounds_add(j, d2, lo2, hi2, bad);
                bounds_add(k, d3, lo3, hi3, bad);
            }
    *had_bad = bad;
    int par[7];
    box_geometry<ORDER, ES>(g, lo1, lo2, lo3, hi1, hi2, hi3, bad, par);
    if (par[3] == 0) return GLOBAL;
    BoxPar bp;
    bp.O1 = par[0]; bp.O2 = par[1]; bp.O3 = par[2];
    bp.E1 = par[3]; bp.E2 = par[4]; bp.E3 = par[5]; bp.S3 = par[6];
    // FP32 box plus the 16-bit staging copy behind it
    const long long floats = static_cast<long long>(bp.E1) * bp.E2 * bp.S3 * (ES == 2 ? 3 : 2) / 2;
    if (floats > kBoxCapFloats || bp.S3 % 32 != 0 || bp.E3 > bp.S3) return BROKEN;
    if (bp.E1 > g.n1 || bp.E2 > g.n2 || bp.E3 > g.n3) return BROKEN;
    const long long P = static_cast<long long>(bp.E2) * bp.S3;
    for (int w = 0; w < TILE2; ++w)
        for (int l = 0; l < TILE3; ++l)
            for (int q = 0; q < TILE1; ++q) {
                const int i = bz * TILE1 + q, j = by * TILE2 + w, k = bx * TILE3 + l;
                if (i >= g.n1 || j >= g.n2 || k >= g.n3) continue;
                float d1, d2, d3, t1, t2, t3;
                disp(i, j, k, d1, d2, d3);
                const int o = tile_offset<ORDER>(bp, i, j, k, d1, d2, d3, t1, t2, t3);
                float u;
                const long long c1 = i + split_in_box(d1, u) - OFF - bp.O1;
                const long long c2 = j + split_in_box(d2, u) - OFF - bp.O2;
                const long long c3 = k + split_in_box(d3, u) - OFF - bp.O3;
                if (c1 < 0 || c1 > bp.E1 - M || c2 < 0 || c2 > bp.E2 - M || c3 < 0 || c3 > bp.E3 - M)
                    return BROKEN;
                if (o != c1 * P + c2 * bp.S3 + c3) return BROKEN;
                // first and last stencil node inside the FP32 box
                const long long last = o + (M - 1) * P + (M - 1) * bp.S3 + (M - 1);
                if (o < 0 || last >= bp.E1 * P) return BROKEN;
                if (!(t1 >= 0.0f && t1 <= 1.0f && t2 >= 0.0f && t2 <= 1.0f && t3 >= 0.0f && t3 <= 1.0f))
                    return BROKEN;
            }
    return FITS;
}

// Run every tile of grid g; `expect_fit` < 0: tiles with a bad displacement
// must take the global path and all others must be consistent; 1: every tile
// must fit the box as well.
template <int ORDER, int ES>
void run_case(const char* name, const Grid& g, const Disp& disp, int expect_fit)
{
    const int bx_n = (g.n3 + TILE3 - 1) / TILE3, by_n = (g.n2 + TILE2 - 1) / TILE2, bz_n = (g.n1 + TILE1 - 1) / TILE1;
    long long fits = 0, glob = 0, bad_tiles = 0;
    for (int bz = 0; bz < bz_n; ++bz)
        for (int by = 0; by < by_n; ++by)
            for (int bx = 0; bx < bx_n; ++bx) {
                bool had_bad = false;
                const Outcome r = run_tile<ORDER, ES>(g, bx, by, bz, disp, &had_bad);
                if (r == BROKEN) {
                    std::printf("FAIL %s (order %d, es %d): tile (%d,%d,%d) box does not hold its stencils\n", name,
                                ORDER, ES, bx, by, bz);
                    ++g_failures;
                    return;
                }
                if (had_bad) {
                    ++bad_tiles;
                    if (r != GLOBAL) {
                        std::printf("FAIL %s (order %d, es %d): tile (%d,%d,%d) with a non-finite or huge "
                                    "displacement was given a shared-memory box\n",
                                    name, ORDER, ES, bx, by, bz);
                        ++g_failures;
                        return;
                    }
                }
                (r == FITS ? fits : glob) += 1;
            }
    if (expect_fit == 1 && glob != 0) {
        std::printf("FAIL %s (order %d, es %d): %lld tiles left the box path\n", name, ORDER, ES, glob);
        ++g_failures;
        return;
    }
    std::printf("ok   %-28s order %d es %d  tiles: %lld box, %lld global (%lld with bad displacements)\n", name,
                ORDER, ES, fits, glob, bad_tiles);
}

// big: the grid is large enough for every tile's box to fit (n3 >= 32 + the
// stencil and spread along x3, likewise along x1 and x2)
template <int ORDER, int ES>
void all_cases(const Grid& g, bool big)
{
    const int fit = big ? 1 : -1;
    const float nan = std::numeric_limits<float>::quiet_NaN();
    const float inf = std::numeric_limits<float>::infinity();
    // smooth displacement of a few cells (a realistic characteristic)
    run_case<ORDER, ES>("smooth", g, [&](int i, int j, int k, float& a, float& b, float& c) {
        a = 1.5f * std::sin(6.2831853f * j / g.n2);
        b = -1.0f * std::cos(6.2831853f * k / g.n3);
        c = 2.0f * std::sin(6.2831853f * i / g.n1);
    }, fit);
    run_case<ORDER, ES>("integer shift", g, [&](int, int, int, float& a, float& b, float& c) {
        a = 3.0f; b = -5.0f; c = 17.0f;
    }, fit);
    run_case<ORDER, ES>("tiny negative", g, [&](int, int, int, float& a, float& b, float& c) {
        a = -1e-9f; b = -1e-30f; c = -0.0f;
    }, fit);
    run_case<ORDER, ES>("all NaN", g, [&](int, int, int, float& a, float& b, float& c) { a = b = c = nan; }, -1);
    run_case<ORDER, ES>("one NaN per tile", g, [&](int i, int j, int k, float& a, float& b, float& c) {
        a = b = c = 0.25f;
        if (i % TILE1 == 1 && j % TILE2 == 3 && k % TILE3 == 7) c = nan;
    }, -1);
    run_case<ORDER, ES>("+Inf", g, [&](int, int, int, float& a, float& b, float& c) { a = inf; b = 0.5f; c = 0.5f; },
                        -1);
    run_case<ORDER, ES>("-Inf", g, [&](int, int, int, float& a, float& b, float& c) { a = 0.5f; b = -inf; c = 0.5f; },
                        -1);
    run_case<ORDER, ES>("+1e7", g, [&](int, int, int, float& a, float& b, float& c) { a = b = c = 1e7f; }, -1);
    run_case<ORDER, ES>("-1e7", g, [&](int, int, int, float& a, float& b, float& c) { a = b = c = -1e7f; }, -1);
    run_case<ORDER, ES>("+2^20", g, [&](int, int, int, float& a, float& b, float& c) {
        a = 0.0f; b = 1048576.0f; c = 0.0f;
    }, -1);
    run_case<ORDER, ES>("just below 2^20", g, [&](int, int, int, float& a, float& b, float& c) {
        a = -1048575.5f; b = 0.0f; c = 1048575.0f;
    }, -1);
    run_case<ORDER, ES>("mixed signs 1e6", g, [&](int i, int j, int k, float& a, float& b, float& c) {
        const float s = ((i + j + k) & 1) ? 1.0f : -1.0f;
        a = s * 1e6f; b = -s * 3e5f; c = s * 999999.0f;
    }, -1);
    std::mt19937 rng(7);
    std::uniform_real_distribution<float> u(-0.5f, 0.5f);
    std::vector<float> r(3u * g.N);
    for (auto& x : r) x = u(rng);
    run_case<ORDER, ES>("random +-0.5", g, [&](int i, int j, int k, float& a, float& b, float& c) {
        const size_t p = (static_cast<size_t>(i) * g.n2 + j) * g.n3 + k;
        a = r[p]; b = r[g.N + p]; c = r[2u * g.N + p];
    }, fit);
    std::uniform_real_distribution<float> wide(-40.0f, 40.0f);
    for (auto& x : r) x = wide(rng);
    run_case<ORDER, ES>("random +-40 (no fit)", g, [&](int i, int j, int k, float& a, float& b, float& c) {
        const size_t p = (static_cast<size_t>(i) * g.n2 + j) * g.n3 + k;
        a = r[p]; b = r[g.N + p]; c = r[2u * g.N + p];
    }, -1);
}

// Every point that passes in_box has all its stencil nodes inside the box.
template <int ORDER>
bool in_box_is_safe(const BoxPar& bp, int i, int j, int k, float d1, float d2, float d3, bool* passed)
{
    constexpr int M = Scheme<ORDER>::M;
    constexpr int OFF = Scheme<ORDER>::OFF;
    *passed = in_box<ORDER>(bp, i, j, k, d1, d2, d3);
    if (!*passed) return true;
    float u;
    const long long c1 = static_cast<long long>(i) + split_in_box(d1, u) - OFF - bp.O1;
    const long long c2 = static_cast<long long>(j) + split_in_box(d2, u) - OFF - bp.O2;
    const long long c3 = static_cast<long long>(k) + split_in_box(d3, u) - OFF - bp.O3;
    if (bp.E1 < M || bp.E2 < M || bp.E3 < M || bp.E3 > bp.S3) return false;
    if (c1 < 0 || c1 > bp.E1 - M || c2 < 0 || c2 > bp.E2 - M || c3 < 0 || c3 > bp.E3 - M) return false;
    const long long P = static_cast<long long>(bp.E2) * bp.S3;
    const long long last = c1 * P + c2 * bp.S3 + c3 + (M - 1) * P + (M - 1) * bp.S3 + (M - 1);
    return last < bp.E1 * P && bp.E1 * P <= kBoxCapFloats;
}

// Table made from field A, gather at field B.  same: B is A, so every point
// of a fitting tile must pass in_box.
template <int ORDER, int ES>
void run_table_case(const char* name, const Grid& g, const Disp& A, const Disp& B, bool same)
{
    const int bx_n = g.n3 / TILE3, by_n = g.n2 / TILE2, bz_n = g.n1 / TILE1;  // exactly tiled grids only
    long long box_tiles = 0, pass = 0, fail_pts = 0;
    for (int bz = 0; bz < bz_n; ++bz)
        for (int by = 0; by < by_n; ++by)
            for (int bx = 0; bx < bx_n; ++bx) {
                int lo1 = INT_MAX, lo2 = INT_MAX, lo3 = INT_MAX, hi1 = INT_MIN, hi2 = INT_MIN, hi3 = INT_MIN;
                bool bad = false;
                for (int w = 0; w < TILE2; ++w)
                    for (int l = 0; l < TILE3; ++l)
                        for (int q = 0; q < TILE1; ++q) {
                            const int i = bz * TILE1 + q, j = by * TILE2 + w, k = bx * TILE3 + l;
                            float d1, d2, d3;
                            A(i, j, k, d1, d2, d3);
                            bounds_add(i, d1, lo1, hi1, bad);
                            bounds_add(j, d2, lo2, hi2, bad);
                            bounds_add(k, d3, lo3, hi3, bad);
                        }
                int par[7];
                box_geometry<ORDER, ES>(g, lo1, lo2, lo3, hi1, hi2, hi3, bad, par);
                if (par[3] == 0) continue;
                ++box_tiles;
                BoxPar bp;
                bp.O1 = par[0]; bp.O2 = par[1]; bp.O3 = par[2];
                bp.E1 = par[3]; bp.E2 = par[4]; bp.E3 = par[5]; bp.S3 = par[6];
                for (int w = 0; w < TILE2; ++w)
                    for (int l = 0; l < TILE3; ++l)
                        for (int q = 0; q < TILE1; ++q) {
                            const int i = bz * TILE1 + q, j = by * TILE2 + w, k = bx * TILE3 + l;
                            float d1, d2, d3;
                            B(i, j, k, d1, d2, d3);
                            bool passed;
                            if (!in_box_is_safe<ORDER>(bp, i, j, k, d1, d2, d3, &passed)) {
                                std::printf("FAIL table %s (order %d, es %d): point (%d,%d,%d) passed in_box with a "
                                            "node outside the box\n", name, ORDER, ES, i, j, k);
                                ++g_failures;
                                return;
                            }
                            (passed ? pass : fail_pts) += 1;
                        }
            }
    if (same && fail_pts != 0) {
        std::printf("FAIL table %s (order %d, es %d): %lld points of fitting tiles failed in_box with their own "
                    "table\n", name, ORDER, ES, fail_pts);
        ++g_failures;
        return;
    }
    std::printf("ok   table %-22s order %d es %d  box tiles %lld, points in box %lld, out %lld\n", name, ORDER, ES,
                box_tiles, pass, fail_pts);
}

// Boxes from arbitrary integer bounds (unordered, extreme, huge) against
// arbitrary displacements: in_box never admits a node outside the box.
template <int ORDER, int ES>
void run_garbage_tables(const Grid& g)
{
    std::mt19937 rng(11);
    std::uniform_int_distribution<int> any(INT_MIN, INT_MAX), near(-10, 74), span(-3, 14), span3(-3, 40);
    std::uniform_real_distribution<float> u(-8.0f, 8.0f);
    const float special[] = {std::numeric_limits<float>::quiet_NaN(), std::numeric_limits<float>::infinity(),
                             -std::numeric_limits<float>::infinity(), 3e9f, -3e9f, 1e7f, -1e7f, 2147483520.0f};
    long long boxes = 0, pass = 0;
    for (int trial = 0; trial < 200000; ++trial) {
        int b[6];
        if (trial % 4 == 0) {  // arbitrary integers
            for (int a = 0; a < 6; ++a) b[a] = any(rng);
        } else {  // plausible but unrelated bounds, sometimes unordered
            for (int a = 0; a < 3; ++a) b[a] = near(rng);
            b[3] = b[0] + span(rng);
            b[4] = b[1] + span(rng);
            b[5] = b[2] + span3(rng);
        }
        int par[7];
        box_geometry<ORDER, ES>(g, b[0], b[1], b[2], b[3], b[4], b[5], false, par);
        if (par[3] == 0) continue;
        ++boxes;
        BoxPar bp;
        bp.O1 = par[0]; bp.O2 = par[1]; bp.O3 = par[2];
        bp.E1 = par[3]; bp.E2 = par[4]; bp.E3 = par[5]; bp.S3 = par[6];
        for (int s = 0; s < 16; ++s) {
            const int i = static_cast<int>(rng() % 64), j = static_cast<int>(rng() % 64),
                      k = static_cast<int>(rng() % 64);
            float d[3];
            for (float& x : d) x = (rng() % 8 == 0) ? special[rng() % 8] : u(rng);
            bool passed;
            if (!in_box_is_safe<ORDER>(bp, i, j, k, d[0], d[1], d[2], &passed)) {
                std::printf("FAIL garbage table (order %d, es %d): bounds %d %d %d %d %d %d, point (%d,%d,%d) + "
                            "(%g,%g,%g) passed in_box outside the box\n", ORDER, ES, b[0], b[1], b[2], b[3], b[4],
                            b[5], i, j, k, d[0], d[1], d[2]);
                ++g_failures;
                return;
            }
            pass += passed;
        }
    }
    std::printf("ok   garbage tables            order %d es %d  fitting boxes %lld, points in box %lld\n", ORDER,
                ES, boxes, pass);
}

template <int ORDER, int ES>
void table_cases(const Grid& g)
{
    const float nan = std::numeric_limits<float>::quiet_NaN();
    const Disp smooth = [&](int i, int j, int k, float& a, float& b, float& c) {
        a = 1.5f * std::sin(6.2831853f * j / g.n2);
        b = -1.0f * std::cos(6.2831853f * k / g.n3);
        c = 2.0f * std::sin(6.2831853f * i / g.n1);
    };
    const Disp other = [&](int i, int j, int k, float& a, float& b, float& c) {
        a = -2.5f * std::cos(6.2831853f * k / g.n3);
        b = 3.0f * std::sin(6.2831853f * i / g.n1);
        c = -1.5f * std::sin(6.2831853f * j / g.n2);
    };
    const Disp bad = [&](int i, int j, int k, float& a, float& b, float& c) {
        smooth(i, j, k, a, b, c);
        if ((i + j + k) % 5 == 0) a = nan;
        if ((i + j + k) % 7 == 0) b = 3e9f;
        if ((i + j + k) % 11 == 0) c = -std::numeric_limits<float>::infinity();
    };
    run_table_case<ORDER, ES>("own field", g, smooth, smooth, true);
    run_table_case<ORDER, ES>("other field", g, smooth, other, false);
    run_table_case<ORDER, ES>("NaN/Inf/huge field", g, smooth, bad, false);
    run_garbage_tables<ORDER, ES>(g);
}

}  // namespace

int main()
{
    // 64^3 and the ragged 70 x 44 x 104 (partial tiles along every axis) hold
    // their boxes; along x3 the small grids are narrower than one box
    const Grid grids[] = {make_grid(64, 64, 64), make_grid(70, 44, 104), make_grid(40, 36, 30),
                          make_grid(16, 24, 8)};
    const bool big[] = {true, true, false, false};
    for (int n = 0; n < 4; ++n) {
        const Grid& g = grids[n];
        std::printf("grid %d x %d x %d\n", g.n1, g.n2, g.n3);
        all_cases<3, 4>(g, big[n]);
        all_cases<1, 4>(g, big[n]);
        all_cases<4, 4>(g, big[n]);
        all_cases<3, 2>(g, big[n]);
        all_cases<1, 2>(g, big[n]);
    }
    const Grid tg = make_grid(64, 64, 64);
    std::printf("tile-bounds tables, grid 64 x 64 x 64\n");
    table_cases<3, 4>(tg);
    table_cases<1, 4>(tg);
    table_cases<4, 4>(tg);
    table_cases<3, 2>(tg);
    table_cases<1, 2>(tg);
    if (g_failures) {
        std::printf("%d case(s) failed\n", g_failures);
        return 1;
    }
    std::printf("OK\n");
    return 0;
}
