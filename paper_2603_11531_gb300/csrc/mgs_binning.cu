// Tile binning without any depth order.
//
// The paper removes depth sorting because the blending sums of Eq. 2 commute
// (Sec. 2, Eq. 1 discussion; Sec. 3.1).  The lists built here are keyed by
// tile only -- a counting sort by tile:
//
//   0. k_group_cost, k_bin_plan: the plan cost of every group of 32
//      consecutive Gaussians (its rectangle rows, each charged kRowCost plus
//      the row's width in tiles) and the exclusive scan of the group costs
//      plus a fixed visit charge.  Every warp of the binning grid (one
//      512-thread CTA per SM) takes an equal contiguous share of that cost
//      numbering, cut at row boundaries.
//   1. k_bin_count: each warp resolves its rows, 32 at a time (one per lane):
//      the tiles of a rectangle row that pass the FP32 tile test form one
//      interval (row_tiles), which is added to a per-CTA shared-memory
//      difference array (+1 at its first tile, -1 after its last); a prefix
//      sum per tile row turns those into the CTA's tile counts, and one
//      global atomicAdd per (CTA, tile) reserves the CTA's block inside the
//      tile and returns its base.
//   2. k_scan_order: exclusive scan of the per-tile totals -> tile offsets,
//      and the rasterisation order (longest lists first).
//   3. k_bin_scatter: the same warps resolve the same rows again and write
//      the rows' tiles (lane by lane, or spread over the warp when a batch
//      holds a long row) at offset[tile] + base[c][tile] + (shared-memory
//      rank).
//
// A pair is listed only if the FP32 tile test (tile_may_hit) allows an
// included pixel in the tile; its rectangle alone (the 3-sigma bounding
// square) would list many tiles a thin ellipse never reaches.  Resolving a
// row costs a handful of test evaluations instead of one per tile (the test
// is monotone along the row up to its vertex, see row_tiles).  Order within a
// tile follows the atomics and is not reproducible; the rasteriser does not
// depend on it beyond FP32 rounding.
#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kScanThreads = 1024;
// Count and scatter run one 512-thread CTA per SM at 64 registers a thread:
// half of the register file, so that the previous frame's rasteriser keeps
// two CTAs on the SM meanwhile.  Alone, 1024 threads per CTA bin faster (count
// 0.051 against 0.068 ms on the 600k benchmark view), but frames in flight on
// several streams render faster this way (971 against 957 FPS).
constexpr int kBinThreads = 512;
constexpr int kBand = 32768;          // words per shared-memory band (128 KB)

__device__ __forceinline__ void rect_of(const uint2 r, int &x0, int &y0, int &w, int &h) {
    x0 = r.x & 0xFFFF;
    y0 = r.y & 0xFFFF;
    w = (int)(r.x >> 16) - x0;
    h = (int)((r.y & ~kRectWide) >> 16) - y0;
}

// FP32-contract tile test: may Gaussian (m, l) include a pixel centre of tile
// (tx, ty)?  Slab bounds at the tile centre with half extent 7.5 and a 2^-18
// relative margin, one correctly rounded operation per step (the oracle
// evaluates the identical sequence, so both build the same lists).  A tile
// that fails holds no pixel with q <= 9.
__device__ __forceinline__ bool tile_may_hit(float mx, float my, float l11, float l21, float l22,
                                             int tx, int ty) {
    const float h = 7.5f;
    const float bx = (float)(tx * kTile + 8), by = (float)(ty * kTile + 8);
    const float dxb = __fsub_rn(bx, mx);
    const float dyb = __fsub_rn(by, my);
    const float e1c = fabsf(__fmaf_rn(l11, dxb, __fmul_rn(l21, dyb)));
    const float h1 = __fmaf_rn(fabsf(l11), h, __fmul_rn(fabsf(l21), h));
    const float u2 = __fadd_rn(fabsf(dyb), h);
    const float s1 = __fadd_rn(__fmul_rn(fabsf(l11), __fadd_rn(fabsf(dxb), h)), __fmul_rn(fabsf(l21), u2));
    const float m1 = __fmul_rn(3.814697265625e-06f, __fadd_rn(s1, 4.0f));
    const float e2c = fabsf(__fmul_rn(l22, dyb));
    const float h2 = __fmul_rn(fabsf(l22), h);
    const float m2 = __fmul_rn(3.814697265625e-06f, __fadd_rn(__fmul_rn(fabsf(l22), u2), 4.0f));
    return __fsub_rn(e1c, h1) <= __fadd_rn(3.0f, m1) && __fsub_rn(e2c, h2) <= __fadd_rn(3.0f, m2);
}

// Row constants of the FP32 tile test for one tile row of one Gaussian:
// along the row only dxb = (tile centre x) - m_x changes.
struct RowTest {
    float mx, l11, P, h1, s12;   // P = l21 dyb, h1 = |l11| h + |l21| h, s12 = |l21| (|dyb| + h)
};
// e1c - h1 of tile tx (left-hand side of the test's first slab)
__device__ __forceinline__ float row_lhs(const RowTest &r, int tx) {
    const float dxb = __fsub_rn((float)(tx * kTile + 8), r.mx);
    return __fsub_rn(fabsf(__fmaf_rn(r.l11, dxb, r.P)), r.h1);
}
// l11 dxb + P of tile tx (its sign changes once along the row)
__device__ __forceinline__ float row_e1(const RowTest &r, int tx) {
    return __fmaf_rn(r.l11, __fsub_rn((float)(tx * kTile + 8), r.mx), r.P);
}
// 3 + m1 for |dxb| = adx (right-hand side of the first slab)
__device__ __forceinline__ float row_rhs(const RowTest &r, float adx) {
    const float s1 = __fadd_rn(__fmul_rn(fabsf(r.l11), __fadd_rn(adx, 7.5f)), r.s12);
    return __fadd_rn(3.0f, __fmul_rn(3.814697265625e-06f, __fadd_rn(s1, 4.0f)));
}
__device__ __forceinline__ int clamp_tile(float v, int lo, int hi) {
    return (int)fminf(fmaxf(v, (float)lo), (float)hi);   // NaN -> lo
}

// Smallest t in [lo, hi] with row_lhs(t) <= K, starting from `guess`; the
// predicate is false ... false true ... true on [lo, hi] and true at hi.
// A few steps from a good guess, else bisection.  *v: row_lhs at the result.
__device__ __forceinline__ int row_first(const RowTest &r, float K, int lo, int hi, int guess,
                                         float &v) {
    int t = min(max(guess, lo), hi);
    v = row_lhs(r, t);
    if (v <= K) {
        for (int s = 0; s < 4 && t > lo; ++s) {
            const float u = row_lhs(r, t - 1);
            if (!(u <= K)) return t;
            --t;
            v = u;
        }
        if (t == lo) return t;
        hi = t;
    } else {
        for (int s = 0; s < 4; ++s) {
            ++t;
            v = row_lhs(r, t);
            if (v <= K) return t;
        }
        lo = t + 1;
    }
    while (lo < hi) {   // bisection on [lo, hi], predicate true at hi
        const int m = (lo + hi) >> 1;
        if (row_lhs(r, m) <= K) hi = m;
        else lo = m + 1;
    }
    v = row_lhs(r, lo);
    return lo;
}
// Largest t in [lo, hi] with row_lhs(t) <= K (true ... true false ... false,
// true at lo).
__device__ __forceinline__ int row_last(const RowTest &r, float K, int lo, int hi, int guess,
                                        float &v) {
    int t = min(max(guess, lo), hi);
    v = row_lhs(r, t);
    if (v <= K) {
        for (int s = 0; s < 4 && t < hi; ++s) {
            const float u = row_lhs(r, t + 1);
            if (!(u <= K)) return t;
            ++t;
            v = u;
        }
        if (t == hi) return t;
        lo = t;
    } else {
        for (int s = 0; s < 4; ++s) {
            --t;
            v = row_lhs(r, t);
            if (v <= K) return t;
        }
        hi = t - 1;
    }
    while (lo < hi) {   // bisection on [lo, hi], predicate true at lo
        const int m = (lo + hi + 1) >> 1;
        if (row_lhs(r, m) <= K) lo = m;
        else hi = m - 1;
    }
    v = row_lhs(r, lo);
    return lo;
}

// The tiles of tile row ty inside rectangle columns [x0, x1) that pass
// tile_may_hit, as one interval [a, b] (a > b: none).  Returns false when it
// cannot establish that they form one interval; the caller then tests every
// tile of the row.
//
// Why an interval: along the row the test is  |l11 dxb + P| - h1 <= 3 + m1
// with dxb = fl(x - m_x).  Every operation is a correctly rounded, hence
// monotone, function of its inputs, so fl(l11 dxb + P) is monotone in the
// tile index, its absolute value falls and then rises, and for any fixed
// bound K the tiles with  fl(|.| - h1) <= K  form an interval.  The margin m1
// grows with |dxb| only, so on the rectangle it lies between its value at
// |dxb| = 0 and its value at the farther end: the tiles passing with the
// larger bound form an interval I_max, those passing with the smaller one an
// interval I_min inside it, and only the tiles of I_max \ I_min (none in
// practice: the bounds differ by 2^-18 relative) are tested one by one.  The
// second slab |l22 dyb| - h2 <= 3 + m2 is the same for the whole row.
// Most rows are settled by a certificate: the two tiles nearest the real
// crossings pass with the smaller bound and their outer neighbours fail with
// the larger one, so I_min = I_max = the tiles between them.
__device__ __forceinline__ bool row_tiles(float mx, float my, float l11, float l21, float l22, int x0,
                                       int x1, int ty, int &a, int &b) {
    a = 1;
    b = 0;
    const float h = 7.5f;
    const float dyb = __fsub_rn((float)(ty * kTile + 8), my);
    const float u2 = __fadd_rn(fabsf(dyb), h);
    const float e2c = fabsf(__fmul_rn(l22, dyb));
    const float h2 = __fmul_rn(fabsf(l22), h);
    const float m2 = __fmul_rn(3.814697265625e-06f, __fadd_rn(__fmul_rn(fabsf(l22), u2), 4.0f));
    if (!(__fsub_rn(e2c, h2) <= __fadd_rn(3.0f, m2))) return true;   // no tile of the row
    RowTest r;
    r.mx = mx;
    r.l11 = l11;
    r.P = __fmul_rn(l21, dyb);
    r.h1 = __fmaf_rn(fabsf(l11), h, __fmul_rn(fabsf(l21), h));
    r.s12 = __fmul_rn(fabsf(l21), u2);
    const int xl = x0, xr = x1 - 1;
    if (!(fabsf(l11) > 0.0f && fabsf(l11) < 3.0e38f && fabsf(r.P) < 3.0e38f && fabsf(mx) < 3.0e38f))
        return false;
    const float Kmin = row_rhs(r, 0.0f);
    const float Kmax = row_rhs(r, fmaxf(fabsf(__fsub_rn((float)(xl * kTile + 8), mx)),
                                        fabsf(__fsub_rn((float)(xr * kTile + 8), mx))));
    // real-valued crossings |l11 dxb + P| = h1 + Kmax around the vertex tz
    const float tz = (mx - 8.0f - r.P / l11) * 0.0625f;
    const float span = (r.h1 + Kmax) / fabsf(l11) * 0.0625f;
    {   // fast path: the tiles gl, gr pass and their outer neighbours fail, so
        // (I_max being an interval) I_max = [gl, gr]
        const int gl = clamp_tile(floorf(tz - span) + 1.0f, xl, xr);
        const int gr = clamp_tile(floorf(tz + span), xl, xr);
        if (gl <= gr) {
            const float vl = row_lhs(r, gl), vr = row_lhs(r, gr);
            const bool out_l = gl == xl || !(row_lhs(r, gl - 1) <= Kmax);
            const bool out_r = gr == xr || !(row_lhs(r, gr + 1) <= Kmax);
            if (vl <= Kmin && vr <= Kmin && out_l && out_r) {   // and I_min = I_max
                a = gl;
                b = gr;
                return true;
            }
        }
    }
    // vertex: the first tile t in [xl, xr + 1] at which l11 dxb + P has the
    // sign of l11 (xr + 1 counts as such); |.| is smallest at t or t - 1
    const float sg = l11 > 0.0f ? 1.0f : -1.0f;
    int t = clamp_tile(floorf(tz) + 1.0f, xl, xr + 1);
    if (t <= xr && row_e1(r, t) * sg >= 0.0f) {
        int s = 0;
        while (t > xl && row_e1(r, t - 1) * sg >= 0.0f) {
            --t;
            if (++s > 8) return false;
        }
    } else {
        int s = 0;
        while (t <= xr && !(row_e1(r, t) * sg >= 0.0f)) {
            ++t;
            if (++s > 8) return false;
        }
    }
    int tm;
    float vm;
    if (t > xr) {
        tm = xr;
        vm = row_lhs(r, xr);
    } else if (t == xl) {
        tm = xl;
        vm = row_lhs(r, xl);
    } else {
        const float v1 = row_lhs(r, t), v0 = row_lhs(r, t - 1);
        tm = v1 <= v0 ? t : t - 1;
        vm = fminf(v1, v0);
    }
    if (!(vm <= Kmax)) return true;   // the lowest point fails even the larger bound
    // I_max from guesses at the real crossings
    float va, vb;
    const int a2 = row_first(r, Kmax, xl, tm, clamp_tile(floorf(tz - span) + 1.0f, xl, tm), va);
    const int b2 = row_last(r, Kmax, tm, xr, clamp_tile(floorf(tz + span), tm, xr), vb);
    if (va <= Kmin && vb <= Kmin) {   // I_min = I_max: every tile of [a2, b2] passes
        a = a2;
        b = b2;
        return true;
    }
    // band tiles: test them one by one; together with I_min they must form one run
    if (b2 - a2 > 64) return false;
    int first = -1, last = -2, runs = 0;
    bool prev = false;
    for (int x = a2; x <= b2; ++x) {
        const float v = row_lhs(r, x);
        const bool p = v <= Kmin || (v <= Kmax && tile_may_hit(mx, my, l11, l21, l22, x, ty));
        if (p && !prev) {
            ++runs;
            if (first < 0) first = x;
        }
        if (p) last = x;
        prev = p;
    }
    if (runs > 1) return false;
    if (runs == 1) {
        a = first;
        b = last;
    }
    return true;
}

// Plan cost of a rectangle row: kRowCost plus one unit per tile of the row.
// The count resolves a row in about the same time whatever its width; the
// scatter also writes the row's listed tiles (about 0.6 of its width).
constexpr int kRowCost = 3;
// Cost of a group in the work plan beyond its rows: a fixed charge for
// visiting it (loading its 32 rectangles, the scans and the row split), so
// that shares over sparse stretches of the scene (many Gaussians with one
// or two rows each) stay short.  Measured on the 600k benchmark view with the
// row certificate: a visit charge of 1024 with a row cost of 3 balanced the
// warps best among 256 ... 1536 and 3 ... 8 (a visit costs about as much as a
// hundred rows).
constexpr int kGroupCost = 1024;

// A lane's Gaussian of a group: rectangle and cull geometry, loaded together
// (the geometry of a Gaussian without a rectangle is loaded but never used),
// one group ahead of its use.
struct GroupLoad {
    uint2 r;
    float4 a;
    float l22;
};
__device__ __forceinline__ GroupLoad load_group(const uint2 *__restrict__ rect,
                                                const ProjRec *__restrict__ rec, int64_t n,
                                                int64_t g0) {
    GroupLoad L{make_uint2(0u, 0u), make_float4(0.f, 0.f, 0.f, 0.f), 0.f};
    const int64_t i = g0 + (threadIdx.x & 31);
    if (i < n) {
        L.r = __ldg(&rect[i]);
        L.a = __ldg(&rec[i].a);
        L.l22 = __ldg(&rec[i].b.x);
    }
    return L;
}

// One row handed to a row callback: Gaussian gid, tile row ty, rectangle
// columns [x0, x1), cull geometry, wide flag.
struct RowItem {
    uint32_t gid;
    int ty, x0, x1;
    float mx, my, l11, l21, l22;
    bool wide;
};

// Rows wait in a per-warp queue in shared memory (kQueue slots)
// until 32 of them fill a batch, so that sparse groups (a few visible
// Gaussians with one or two rows) still give every lane a row.
constexpr int kQueue = 64;

// A queued row: {gid, ty | wide << 31, x0 | x1 << 16, l22} and {m_x, m_y, l11, l21}.
struct RowSlot {
    uint4 u;
    float4 g;
};

// Calls f(active, item) with queued rows [qh, qh + cnt) (cnt <= 32), one per
// lane; every lane calls f.
template <class F>
__device__ __forceinline__ void run_rows(const RowSlot *q, int qh, int cnt, F &&f) {
    const int lane = threadIdx.x & 31;
    RowItem it{};
    const bool active = lane < cnt;
    if (active) {
        const RowSlot e = q[(qh + lane) & (kQueue - 1)];
        it.gid = e.u.x;
        it.ty = (int)(e.u.y & 0x7FFFFFFFu);
        it.wide = (e.u.y >> 31) != 0u;
        it.x0 = (int)(e.u.z & 0xFFFFu);
        it.x1 = (int)(e.u.z >> 16);
        it.l22 = __uint_as_float(e.u.w);
        it.mx = e.g.x;
        it.my = e.g.y;
        it.l11 = e.g.z;
        it.l21 = e.g.w;
    }
    f(active, it);
}

// Queues the rows of the group at g0 (Gaussians g0 .. g0 + 31, one per lane)
// whose start cost lies in [ca, cb) of the group's row cost numbering
// (Gaussian after Gaussian, rows top to bottom, row k of Gaussian i starting
// at cost excl_i + k (kRowCost + w_i)), and runs every full batch of 32.
template <class F>
__device__ __forceinline__ void warp_rows(const GroupLoad &L, int64_t g0, int ca, int cb,
                                          RowSlot *q, int &qh, int &qn, F &&f) {
    const int lane = threadIdx.x & 31;
    int x0 = 0, y0 = 0, w = 0, h = 0;
    rect_of(L.r, x0, y0, w, h);
    const bool wide = (L.r.y & kRectWide) != 0;
    const int rc = kRowCost + w;
    const int c = (w > 0 && h > 0) ? h * rc : 0;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - c;
    // rows k with ca <= excl + k rc < cb
    int r0 = 0, nr = 0;
    if (c > 0) {
        r0 = ca > excl ? (ca - excl + rc - 1) / rc : 0;
        const int r1 = cb >= incl ? h : (cb > excl ? min((cb - excl + rc - 1) / rc, h) : 0);
        nr = max(r1 - r0, 0);
    }
    int rincl = nr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, rincl, o);
        if (lane >= o) rincl += y;
    }
    const int rexcl = rincl - nr;
    const int R = __shfl_sync(0xffffffffu, rincl, 31);
    const int ybase = y0 + r0 - rexcl;   // row of index p for this lane: ybase + p
    for (int base = 0; base < R; base += 32) {
        const int p = base + lane;
        // owner: the largest lane whose exclusive prefix is <= p
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(0xffffffffu, rexcl, lo + step);
            if (e <= p) lo += step;
        }
        const int ty = __shfl_sync(0xffffffffu, ybase, lo) + p;
        const uint32_t xw = __shfl_sync(0xffffffffu, (uint32_t)x0 | ((uint32_t)(x0 + w) << 16) |
                                                         (wide ? 0x80000000u : 0u), lo);
        RowSlot e;
        e.u = make_uint4((uint32_t)(g0 + lo), (uint32_t)ty | (xw & 0x80000000u), xw & 0x7FFFFFFFu,
                         __float_as_uint(__shfl_sync(0xffffffffu, L.l22, lo)));
        e.g = make_float4(__shfl_sync(0xffffffffu, L.a.x, lo), __shfl_sync(0xffffffffu, L.a.y, lo),
                          __shfl_sync(0xffffffffu, L.a.z, lo), __shfl_sync(0xffffffffu, L.a.w, lo));
        if (p < R) q[(qh + qn + lane) & (kQueue - 1)] = e;
        __syncwarp();
        qn += min(32, R - base);
        if (qn >= 32) {
            run_rows(q, qh, 32, f);
            qh = (qh + 32) & (kQueue - 1);
            qn -= 32;
            __syncwarp();
        }
    }
}

// Largest group g with cexcl[g] <= c (c < cexcl[groups]).
__device__ __forceinline__ int64_t find_group(const unsigned long long *__restrict__ cexcl,
                                              int64_t groups, unsigned long long c) {
    int64_t lo = 0, hi = groups - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (cexcl[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Calls f(active, item) for the rows of this warp's share of the work plan:
// group g occupies costs [cexcl[g], cexcl[g + 1]), its visit charge first and
// then its row costs; warp w of W takes costs [C w / W, C (w + 1) / W) of the
// total C, and a row belongs to the share holding its start cost.  The plan
// entries are read 32 at a time and groups without rows (all Gaussians
// culled) are skipped without loading them; each group with rows is loaded
// while the previous one is processed.
template <class F>
__device__ __forceinline__ void warp_share_rows(const uint2 *__restrict__ rect,
                                                const ProjRec *__restrict__ rec, int64_t n,
                                                const unsigned long long *__restrict__ cexcl,
                                                int64_t groups, RowSlot *q, F &&f) {
    if (groups == 0) return;
    const int lane = threadIdx.x & 31;
    int qh = 0, qn = 0;   // queued rows: slots [qh, qh + qn) mod kQueue
    const unsigned long long C = cexcl[groups];
    const unsigned long long W = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const unsigned long long c0 = C * w / W, c1 = C * (w + 1) / W;
    if (c0 >= c1) return;
    for (int64_t gb = find_group(cexcl, groups, c0); gb < groups; gb += 32) {
        const int64_t gl = gb + lane;
        const unsigned long long e0l = gl < groups ? cexcl[gl] : C;
        const unsigned long long e1l = gl < groups ? cexcl[gl + 1] : C;
        // groups of this chunk with rows whose row costs meet [c0, c1)
        unsigned m = __ballot_sync(0xffffffffu, gl < groups && e1l - e0l > (unsigned long long)kGroupCost &&
                                                    e1l > c0 && e0l + kGroupCost < c1);
        const bool done = __ballot_sync(0xffffffffu, gl >= groups || e1l >= c1) != 0u;
        if (m) {
            int j = __ffs(m) - 1;
            m &= m - 1;
            GroupLoad cur = load_group(rect, rec, n, (gb + j) * 32);
            for (;;) {
                const int jn = m ? __ffs(m) - 1 : -1;
                GroupLoad nxt{};
                if (jn >= 0) nxt = load_group(rect, rec, n, (gb + jn) * 32);   // in flight meanwhile
                const unsigned long long e0 = __shfl_sync(0xffffffffu, e0l, j);
                const unsigned long long e1 = __shfl_sync(0xffffffffu, e1l, j);
                const long long nc = (long long)(e1 - e0) - kGroupCost;    // row costs of the group
                const long long ca = max(0ll, (long long)(c0 > e0 ? c0 - e0 : 0ull) - kGroupCost);
                const long long cb = min(nc, (long long)(c1 - e0) - kGroupCost);
                if (ca < cb) warp_rows(cur, (gb + j) * 32, (int)ca, (int)cb, q, qh, qn, f);
                if (jn < 0) break;
                j = jn;
                m &= m - 1;
                cur = nxt;
            }
        }
        if (done) break;
    }
    if (qn > 0) run_rows(q, qh, qn, f);
}

// Plan cost of every group of 32 consecutive Gaussians: the sum of
// h (kRowCost + w) over its rectangles (one warp per group).
__global__ void __launch_bounds__(kBinThreads) k_group_cost(const uint2 *__restrict__ rect,
                                                            int64_t n, uint32_t *__restrict__ grp) {
    const int64_t g = ((int64_t)blockIdx.x * kBinThreads + threadIdx.x) >> 5;
    const int64_t i = g * 32 + (threadIdx.x & 31);
    uint32_t c = 0;
    if (i < n) {
        int x0, y0, w, h;
        rect_of(rect[i], x0, y0, w, h);
        c = (w > 0 && h > 0) ? (uint32_t)(h * (kRowCost + w)) : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && g * 32 < n) grp[g] = c;
}

// Exclusive scan of the group costs (plus kGroupCost) into cexcl[0..groups]
// (64-bit), by one block, kPlanSeg groups at a time staged in shared memory
// so that global loads and stores stay coalesced.
constexpr int kPlanSeg = 16384;   // 64-bit costs per pass
// Shared-memory slot of entry i: one pad word every 16 entries, so that
// threads scanning runs of 16 consecutive entries hit different banks.
__device__ __forceinline__ int plan_slot(int i) { return i + (i >> 4); }
constexpr int kPlanSlots = kPlanSeg + kPlanSeg / 16;
__global__ void __launch_bounds__(kScanThreads) k_bin_plan(const uint32_t *__restrict__ grp,
                                                           int64_t groups,
                                                           unsigned long long *__restrict__ cexcl) {
    extern __shared__ unsigned long long seg[];
    __shared__ unsigned long long warp_sums[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long carry = 0;   // identical in every thread
    for (int64_t s0 = 0; s0 < groups; s0 += kPlanSeg) {
        const int m = (int)(groups - s0 < kPlanSeg ? groups - s0 : kPlanSeg);
        for (int i = tid; i < m; i += kScanThreads)
            seg[plan_slot(i)] = (unsigned long long)grp[s0 + i] + kGroupCost;
        __syncthreads();
        const int per = (m + kScanThreads - 1) / kScanThreads;
        const int lo = min(tid * per, m), hi = min(lo + per, m);
        unsigned long long local = 0;
        for (int i = lo; i < hi; ++i) local += seg[plan_slot(i)];
        unsigned long long incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_sums[lane] = t;
        }
        __syncthreads();
        unsigned long long run = carry + (incl - local) + (warp > 0 ? warp_sums[warp - 1] : 0ull);
        for (int i = lo; i < hi; ++i) {
            const unsigned long long v = seg[plan_slot(i)];
            seg[plan_slot(i)] = run;
            run += v;
        }
        carry += warp_sums[kScanThreads / 32 - 1];
        __syncthreads();
        for (int i = tid; i < m; i += kScanThreads) cexcl[s0 + i] = seg[plan_slot(i)];
        __syncthreads();
    }
    if (tid == 0) cexcl[groups] = carry;
}

// Tile rows per shared-memory band: the count's difference array takes
// tiles_x + 1 words per tile row.
__host__ __device__ __forceinline__ int band_rows(int tiles_x, int tiles_y) {
    const int r = kBand / (tiles_x + 1);
    return r < tiles_y ? r : tiles_y;
}

// Counts per tile; with `tc` (tensor-core rasteriser) and a frame that has
// wide Gaussians, also sets kTileWide in tile_count[] of every tile that
// lists one (per-CTA counts stay below 2^31, so the flag never meets a carry).
// Shared memory: the band's difference array (band_rows x (tiles_x + 1)
// ints), then one wide-flag byte per tile of the band.
__global__ void __launch_bounds__(kBinThreads, 2) k_bin_count(const uint2 *__restrict__ rect,
                                                           const ProjRec *__restrict__ rec,
                                                           int64_t n, int tiles_x, int tiles_y,
                                                           const unsigned long long *__restrict__ excl,
                                                           int64_t groups,
                                                           uint32_t *__restrict__ tile_count,
                                                           uint32_t *__restrict__ bases,
                                                           const DevStatus *__restrict__ status,
                                                           bool tc) {
    extern __shared__ int diff_s[];
    __shared__ RowSlot queue_s[kBinThreads / 32][kQueue];
    const int T = tiles_x * tiles_y;
    const int stride = tiles_x + 1;
    const int brows = band_rows(tiles_x, tiles_y);
    unsigned char *wide_s = reinterpret_cast<unsigned char *>(diff_s + brows * stride);
    const bool mark = tc && status->wide_bits != 0u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ty0 = 0; ty0 < tiles_y; ty0 += brows) {
        const int nrows = min(brows, tiles_y - ty0);
        for (int i = threadIdx.x; i < nrows * stride; i += kBinThreads) diff_s[i] = 0;
        if (mark)
            for (int i = threadIdx.x; i < nrows * tiles_x; i += kBinThreads) wide_s[i] = 0;
        __syncthreads();
        warp_share_rows(rect, rec, n, excl, groups, queue_s[warp], [&](bool active, const RowItem &it) {
            const int ry = it.ty - ty0;
            if (!active || (unsigned)ry >= (unsigned)nrows) return;
            int *d = diff_s + ry * stride;
            int a, b;
            if (row_tiles(it.mx, it.my, it.l11, it.l21, it.l22, it.x0, it.x1, it.ty, a, b)) {
                if (a <= b) {
                    atomicAdd(&d[a], 1);
                    atomicAdd(&d[b + 1], -1);
                    if (mark && it.wide)
                        for (int x = a; x <= b; ++x) wide_s[ry * tiles_x + x] = 1;
                }
            } else {   // not one interval: every tile of the row on its own
                for (int x = it.x0; x < it.x1; ++x)
                    if (tile_may_hit(it.mx, it.my, it.l11, it.l21, it.l22, x, it.ty)) {
                        atomicAdd(&d[x], 1);
                        atomicAdd(&d[x + 1], -1);
                        if (mark && it.wide) wide_s[ry * tiles_x + x] = 1;
                    }
            }
        });
        __syncthreads();
        // prefix sums along each tile row -> this CTA's tile counts; reserve
        // the CTA's block in every tile it lists pairs in
        for (int ry = warp; ry < nrows; ry += kBinThreads / 32) {
            int carry = 0;
            for (int xb = 0; xb < tiles_x; xb += 32) {
                const int x = xb + lane;
                int v = x < tiles_x ? diff_s[ry * stride + x] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += y;
                }
                const int c = carry + v;
                carry += __shfl_sync(0xffffffffu, v, 31);
                if (x < tiles_x) {
                    const int t = (ty0 + ry) * tiles_x + x;
                    if (c > 0)
                        bases[(int64_t)blockIdx.x * T + t] =
                            atomicAdd(&tile_count[t], (uint32_t)c) & kTileMask;
                    if (mark && wide_s[ry * tiles_x + x]) atomicOr(&tile_count[t], kTileWide);
                }
            }
        }
        __syncthreads();
    }
}

// Rows of at most this many listed tiles are written lane by lane; a batch
// holding a longer one spreads its tiles over the warp instead.
constexpr int kLaneRun = 16;

__global__ void __launch_bounds__(kBinThreads, 2) k_bin_scatter(
    const uint2 *__restrict__ rect, int64_t n, int tiles_x, int tiles_y,
    const unsigned long long *__restrict__ excl, int64_t groups,
    const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ bases,
    uint32_t *__restrict__ gids, uint64_t capacity, const DevStatus *__restrict__ status,
    const ProjRec *__restrict__ rec, uint4 *__restrict__ wt16) {
    extern __shared__ uint32_t cur_s[];
    __shared__ RowSlot queue_s[kBinThreads / 32][kQueue];
    if (status->last_pairs > capacity) return;  // overflow: lists are not built
    const int we = (int)((status->wmax_frame_bits >> 23) & 0xFFu) - 127;
    if (wt16 && we >= 14) {   // preprocessing wrote the FP16 weights unscaled; rescale them
        const float scale = __int_as_float((127 + 14 - we) << 23);
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
             g += (int64_t)gridDim.x * blockDim.x) {
            const uint2 r = rect[g];
            if (r.x | r.y) wt16[g] = weights_f16(rec[g], scale);
        }
    }
    const int T = tiles_x * tiles_y;
    const int brows = band_rows(tiles_x, tiles_y);
    const int lane = threadIdx.x & 31;
    for (int ty0 = 0; ty0 < tiles_y; ty0 += brows) {
        const int nrows = min(brows, tiles_y - ty0);
        const int t0 = ty0 * tiles_x, bn = nrows * tiles_x;
        // entries of tiles this CTA has no pairs in are never read
        for (int i = threadIdx.x; i < bn; i += kBinThreads)
            cur_s[i] = offsets[t0 + i] + bases[(int64_t)blockIdx.x * T + t0 + i];
        __syncthreads();
        warp_share_rows(rect, rec, n, excl, groups, queue_s[threadIdx.x >> 5], [&](bool active, const RowItem &it) {
            const int ry = it.ty - ty0;
            const bool in = active && (unsigned)ry < (unsigned)nrows;
            int a = 1, b = 0;
            const bool one = in ? row_tiles(it.mx, it.my, it.l11, it.l21, it.l22, it.x0, it.x1,
                                            it.ty, a, b)
                                : true;
            const int L = (in && one && a <= b) ? b - a + 1 : 0;
            if (__reduce_max_sync(0xffffffffu, (unsigned)L) <= (unsigned)kLaneRun) {
                // short rows: each lane writes its own row's tiles
                for (int x = a; x < a + L; ++x) {
                    const uint32_t slot = atomicAdd(&cur_s[ry * tiles_x + x], 1u);
                    if (slot < capacity) gids[slot] = it.gid;
                }
            } else {
                // a long row among them: the rows' tiles, 32 at a time over the warp
                int incl = L;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int ex = incl - L;
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                const int tb = ry * tiles_x + a - ex;   // band tile of pair p of this lane: tb + p
                for (int base = 0; base < total; base += 32) {
                    const int p = base + lane;
                    int lo = 0;   // owner: the largest lane whose exclusive prefix is <= p
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int e = __shfl_sync(0xffffffffu, ex, lo + step);
                        if (e <= p) lo += step;
                    }
                    const int t = __shfl_sync(0xffffffffu, tb, lo) + p;
                    const uint32_t gid = __shfl_sync(0xffffffffu, it.gid, lo);
                    if (p < total) {
                        const uint32_t slot = atomicAdd(&cur_s[t], 1u);
                        if (slot < capacity) gids[slot] = gid;
                    }
                }
            }
            if (in && !one)   // not one interval: every tile of the row on its own
                for (int x = it.x0; x < it.x1; ++x)
                    if (tile_may_hit(it.mx, it.my, it.l11, it.l21, it.l22, x, it.ty)) {
                        const uint32_t slot = atomicAdd(&cur_s[ry * tiles_x + x], 1u);
                        if (slot < capacity) gids[slot] = it.gid;
                    }
        });
        __syncthreads();
    }
}

// One block over the per-tile totals:
//   * exclusive scan of tile_count[T] into tile_offsets[T+1]; records the
//     pair count and flags capacity overflow;
//   * rasterisation order: tiles by decreasing list length (bucketed by
//     floor(log2(length))), so the longest tiles start first and the tail of
//     the raster launch is made of short tiles;
//   * hands this frame's weight bound to the rasteriser and resets the
//     accumulator (and the wide-Gaussian flag) for the next frame;
//   * carries each tile's kTileWide flag from tile_count[] into its order
//     entry.
__global__ void __launch_bounds__(kScanThreads) k_scan_order(const uint32_t *__restrict__ count,
                                                             uint32_t *__restrict__ offsets,
                                                             uint32_t *__restrict__ order, int T,
                                                             uint64_t capacity, DevStatus *status) {
    __shared__ unsigned long long warp_sums[kScanThreads / 32];
    __shared__ unsigned long long carry;
    __shared__ uint32_t hist[33], start[33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        carry = 0;
        status->wmax_frame_bits = status->wmax_bits;
        status->wmax_bits = 0u;
        status->wide_bits = 0u;
        status->last_visible = status->visible;
        status->visible = 0u;
        status->last_wide_tiles = 0u;
    }
    if (tid < 33) hist[tid] = 0u;
    __syncthreads();
    for (int base = 0; base < T; base += kScanThreads * 4) {
        const int i0 = base + tid * 4;
        unsigned long long v[4], local = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (i0 + k < T) ? (count[i0 + k] & kTileMask) : 0u;
            local += v[k];
            if (i0 + k < T) {
                const uint32_t c = (uint32_t)v[k];
                atomicAdd(&hist[c ? 32 - __clz(c) : 0], 1u);   // bucket 0 (empty) .. 32
            }
        }
        unsigned long long incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long sw = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, sw, o);
                if (lane >= o) sw += y;
            }
            warp_sums[lane] = sw;
        }
        __syncthreads();
        unsigned long long run = carry + (incl - local) + (warp > 0 ? warp_sums[warp - 1] : 0ull);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < T) offsets[i0 + k] = (uint32_t)run;
            run += v[k];
        }
        __syncthreads();
        if (tid == kScanThreads - 1) carry = run;
        __syncthreads();
    }
    if (tid == 0) {
        const unsigned long long K = carry;
        offsets[T] = (uint32_t)K;
        status->last_pairs = K;
        atomicMax(&status->max_pairs, K);
        if (K > capacity || K > 0xFFFFFFFFull) atomicOr(&status->overflow, kStatusOverflow);
        uint32_t r = 0;
        for (int bk = 32; bk >= 0; --bk) {      // longest bucket first
            start[bk] = r;
            r += hist[bk];
        }
    }
    __syncthreads();
    for (int t = tid; t < T; t += blockDim.x) {
        const uint32_t cw = count[t], c = cw & kTileMask;
        order[atomicAdd(&start[c ? 32 - __clz(c) : 0], 1u)] = (uint32_t)t | (cw & kTileWide);
        if (cw & kTileWide) atomicAdd(&status->last_wide_tiles, 1u);
    }
}

}  // namespace

// One binning CTA per SM at most (one per 1024 Gaussians below that): the
// work plan balances the warps, so a second resident CTA would only add
// per-CTA tile bases.
int bin_ctas(int64_t n, int sm_count) {
    int64_t c = (n + 1023) / 1024;
    const int64_t cap = (int64_t)sm_count;
    if (c > cap) c = cap;
    return c < 1 ? 1 : (int)c;
}

int64_t bin_scratch_words(int64_t n, int64_t T, int sm_count) {
    return bin_scratch_words_for(bin_ctas(n, sm_count), T, n);
}

cudaError_t launch_binning(const RenderArgs &a, int sm_count, uint32_t *scratch,
                           cudaStream_t stream, const cudaEvent_t *marks) {
    const int tx = a.cam.tiles_x, ty = a.cam.tiles_y;
    const int T = tx * ty;
    const int C = bin_ctas(a.n, sm_count);
    const int64_t groups = (a.n + 31) / 32;
    uint32_t *bases = scratch;
    unsigned long long *excl =
        reinterpret_cast<unsigned long long *>(scratch + ((int64_t)C * T + 1) / 2 * 2);
    uint32_t *grp = reinterpret_cast<uint32_t *>(excl + groups + 1);
    const int brows = band_rows(tx, ty);
    const size_t count_smem = ((size_t)brows * (tx + 1) * sizeof(int) + (size_t)brows * tx + 15) / 16 * 16;
    const size_t scatter_smem = (size_t)brows * tx * sizeof(uint32_t);
    cudaError_t e = cudaMemsetAsync(a.tile_count, 0, (size_t)T * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    if (a.n > 0) {
        if ((e = cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kBand * (sizeof(int) + 1)))) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kBand * sizeof(uint32_t)))) != cudaSuccess)
            return e;
        k_group_cost<<<(int)((groups * 32 + kBinThreads - 1) / kBinThreads), kBinThreads, 0,
                       stream>>>(a.rect, a.n, grp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int plan_n = (int)(groups < kPlanSeg ? groups : kPlanSeg);
        const size_t plan_smem = (size_t)(plan_n + plan_n / 16) * sizeof(unsigned long long);
        if ((e = cudaFuncSetAttribute(k_bin_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kPlanSlots * sizeof(unsigned long long)))) != cudaSuccess)
            return e;
        k_bin_plan<<<1, kScanThreads, plan_smem, stream>>>(grp, groups, excl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (marks && (e = cudaEventRecord(marks[0], stream)) != cudaSuccess) return e;
        k_bin_count<<<C, kBinThreads, count_smem, stream>>>(a.rect, a.rec, a.n, tx, ty, excl, groups,
                                                            a.tile_count, bases, a.status,
                                                            tc_raster(a));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (marks && (e = cudaEventRecord(marks[1], stream)) != cudaSuccess) return e;
    } else if (marks) {
        if ((e = cudaEventRecord(marks[0], stream)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(marks[1], stream)) != cudaSuccess) return e;
    }
    k_scan_order<<<1, kScanThreads, 0, stream>>>(a.tile_count, a.tile_offsets, a.tile_order, T,
                                                 a.capacity, a.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (marks && (e = cudaEventRecord(marks[2], stream)) != cudaSuccess) return e;
    if (a.n == 0) return e;
    k_bin_scatter<<<C, kBinThreads, scatter_smem, stream>>>(a.rect, a.n, tx, ty, excl, groups,
                                                            a.tile_offsets, bases, a.gids,
                                                            a.capacity, a.status, a.rec,
                                                            tc_raster(a) ? a.wt16 : nullptr);
    return cudaGetLastError();
}

}  // namespace mgs
