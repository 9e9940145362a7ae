// bsp_api.cu -- the C ABI of libbsp (include/bsp.h): plan creation, argument
// checks, workspace layout, scheduling of the contraction tiles, and the
// host orchestration of filter -> inverse FFT -> contraction -> reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "../../include/bsp.h"
#include "bsp_internal.h"

using namespace bsp;

namespace {

thread_local std::string g_last_error;
constexpr int CCOLS = 64;   // pairs per CUDA-core contraction tile (bsp_contract.cu)

bsp_status cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return BSP_ECUDA;
}
}  // namespace

bsp_status bsp::record_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }

namespace {

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }
size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Radix stages for an inverse DFT of length m (8s first, then 4, 2, 3, 5).
bool radix_plan(int m, int* rad, int* nrad) {
    int a = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    std::vector<int> r;
    int n8 = a / 3, rem = a % 3;
    if (rem == 1 && n8 > 0) { --n8; r.push_back(4); r.push_back(4); }
    else if (rem == 1) r.push_back(2);
    else if (rem == 2) r.push_back(4);
    for (int i = 0; i < n8; ++i) r.insert(r.begin(), 8);
    while (m % 3 == 0) { m /= 3; r.push_back(3); }
    while (m % 5 == 0) { m /= 5; r.push_back(5); }
    if (m != 1 || (int)r.size() > 8) return false;
    *nrad = (int)r.size();
    for (size_t i = 0; i < r.size(); ++i) rad[i] = r[i];
    return true;
}

struct DevSched {
    Work* works = nullptr;
    int2* pairs = nullptr;
    int* rowf = nullptr;
    BinLoc* loc = nullptr;
    int nwork = 0, npair = 0, nrowf = 0, nloc = 0, nsplit = 1;
    void release() {
        cudaFree(works); cudaFree(pairs); cudaFree(rowf); cudaFree(loc);
        works = nullptr; pairs = nullptr; rowf = nullptr; loc = nullptr;
    }
};

struct HostSched {
    std::vector<Work> works;
    std::vector<int2> pairs;
    std::vector<int> rowf;
    std::vector<BinLoc> loc;   // [nslots_out][nbins]
    int nsplit = 1;
};

typedef std::vector<std::array<int, 3>> BinList;

// Every distinct (a; b >= c) whose shells form one of the sorted bins, in
// lexicographic order: the Legendre leg on each of the three shells in turn.
BinList expand_full(const BinList& sorted) {
    std::map<std::array<int, 3>, int> m;
    for (const auto& t : sorted)
        for (int k = 0; k < 3; ++k) {
            const int a = t[k], u = t[(k + 1) % 3], v = t[(k + 2) % 3];
            m[{a, std::max(u, v), std::min(u, v)}] = 1;
        }
    BinList out;
    for (auto& kv : m) out.push_back(kv.first);
    return out;
}

// Tiles of <= `cols` pairs (b, c) (sorted by b, then c; the shells they touch
// span <= 64), each with the rows (slot, a) for a in the tile's a-range, cut
// into chunks of <= 64 rows.
HostSched build_sched(const BinList& bins, const std::vector<int>& out_slots, int nsh, size_t npts,
                      int target_ctas, int cols) {
    HostSched h;
    std::map<std::pair<int, int>, int> pidx;
    for (auto& t : bins) pidx[{t[1], t[2]}] = 0;
    std::vector<std::pair<int, int>> pl;
    for (auto& kv : pidx) pl.push_back(kv.first);   // sorted by (b, c)
    // per pair: a-range
    std::vector<int> alo(pl.size(), 1 << 30), ahi(pl.size(), -1);
    for (size_t i = 0; i < pl.size(); ++i) pidx[pl[i]] = (int)i;
    for (auto& t : bins) {
        int p = pidx[{t[1], t[2]}];
        alo[p] = std::min(alo[p], t[0]);
        ahi[p] = std::max(ahi[p], t[0]);
    }
    struct TileInfo { int p0, np, alo, ahi, rowbase_chunk0, work0; };
    std::vector<TileInfo> tiles;
    size_t i = 0;
    while (i < pl.size()) {
        int p0 = (int)i, slo = pl[i].second, shi = pl[i].first, lo = alo[i], hi = ahi[i];
        size_t j = i + 1;
        while (j < pl.size() && (int)(j - i) < cols) {
            int nslo = std::min(slo, pl[j].second), nshi = std::max(shi, pl[j].first);
            if (nshi - nslo + 1 > 64) break;
            slo = nslo; shi = nshi;
            lo = std::min(lo, alo[j]); hi = std::max(hi, ahi[j]);
            ++j;
        }
        TileInfo ti{p0, (int)(j - i), lo, hi, 0, (int)h.works.size()};
        int na = hi - lo + 1, nrows = na * (int)out_slots.size();
        for (int r0 = 0; r0 < nrows; r0 += 64) {
            Work w{};
            w.pair0 = p0; w.npairs = (int)(j - i);
            w.row0 = r0; w.nrows = std::min(64, nrows - r0);
            w.rowbase = (int)h.rowf.size();
            w.shell_lo = slo; w.nshell = shi - slo + 1;
            for (int r = r0; r < r0 + w.nrows; ++r) {
                int si = r / na, a = lo + r % na;
                h.rowf.push_back(out_slots[si] * nsh + a);
            }
            h.works.push_back(w);
        }
        tiles.push_back(ti);
        i = j;
    }
    for (auto& p : pl) h.pairs.push_back(int2{p.first, p.second});
    // pair -> tile
    std::vector<int> tile_of(pl.size());
    for (size_t t = 0; t < tiles.size(); ++t)
        for (int p = tiles[t].p0; p < tiles[t].p0 + tiles[t].np; ++p) tile_of[p] = (int)t;
    h.loc.resize(out_slots.size() * bins.size());
    for (size_t si = 0; si < out_slots.size(); ++si)
        for (size_t b = 0; b < bins.size(); ++b) {
            int p = pidx[{bins[b][1], bins[b][2]}];
            const TileInfo& ti = tiles[tile_of[p]];
            int na = ti.ahi - ti.alo + 1;
            int row = (int)si * na + (bins[b][0] - ti.alo);
            BinLoc L{ti.work0 + row / 64, row % 64, p - ti.p0, 0};
            h.loc[si * bins.size() + b] = L;
        }
    int nw = std::max<int>(1, (int)h.works.size());
    long long by_len = (long long)((npts + 8191) / 8192);
    long long by_ctas = (target_ctas + nw - 1) / nw;
    h.nsplit = (int)std::max<long long>(1, std::min(by_len, by_ctas));
    return h;
}

template <typename T>
bsp_status upload(T** dst, const std::vector<T>& v) {
    *dst = nullptr;
    if (v.empty()) return BSP_OK;
    CK(cudaMalloc((void**)dst, sizeof(T) * v.size()));
    CK(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return BSP_OK;
}

bsp_status upload_sched(DevSched& d, const HostSched& h) {
    d.release();
    bsp_status s;
    if ((s = upload(&d.works, h.works)) != BSP_OK) return s;
    if ((s = upload(&d.pairs, h.pairs)) != BSP_OK) return s;
    if ((s = upload(&d.rowf, h.rowf)) != BSP_OK) return s;
    if ((s = upload(&d.loc, h.loc)) != BSP_OK) return s;
    d.nwork = (int)h.works.size();
    d.npair = (int)h.pairs.size();
    d.nrowf = (int)h.rowf.size();
    d.nloc = (int)h.loc.size();
    d.nsplit = h.nsplit;
    return BSP_OK;
}

size_t partial_bytes(const HostSched& h, int cols) {
    return (size_t)h.works.size() * h.nsplit * 64 * cols * sizeof(double);
}

// Tensor-core schedule: tiles of <= 128 pairs (sorted by (b, c), shells
// spanned <= 64); each tile's rows are the fields (slot, a) for a in the
// tile's a-range, in boxes of 8 consecutive fields, <= 16 boxes (N <= 128)
// per work item.
struct TcSched {
    std::vector<TcWork> works;
    std::vector<int2> pairs;
    std::vector<BinLoc> loc;
    std::vector<TcUnit> units;
    int lsup = 1, nsup = 1;
};

// Persistent units: each work gets CTAs in proportion to its cost per
// K-block, all CTAs together about one per SM; every super-segment of lsup
// K-blocks is split among the work's CTAs, so all works sweep x in the same
// order at about the same rate and read the same fields while they are in
// L2.  Nothing holds the CTAs together: a global counter that made every CTA
// wait for the others at each super-segment (any allowed drift, 1 to 16
// super-segments) cost 6 % at 512^3 against letting them run (224 -> 210 ms),
// the acquire load on the contended counter sitting in the copy thread's
// path.  The cost of a K-block is set by the warps' hand-offs and hardly
// depends on the MMA N (clock traces on GB300: ~1 700 to 1 800 busy cycles per
// K-block for N = 32 and N = 96 alike), so the weight is almost flat in N;
// weighting by N, as the first versions did, gave works of small N 1.9x the
// K-blocks per CTA.  With whole CTAs per work the split is uneven when the
// works do not divide the SMs (17 works on 152 SMs at 512^3: one work of 8
// CTAs, whose CTAs run 12.5 % longer).  Equal shares with a CTA running the
// tail of one work and then the head of the next were slower (205 -> 219 ms):
// the second unit starts where the other CTAs of its work passed long ago
// and reads its fields from DRAM instead of L2.
void assign_units(TcSched& h, size_t npts, int nsm) {
    const int nw = (int)h.works.size();
    const long long nkb = (long long)((npts + 63) / 64);
    const int maxc = (int)std::max<long long>(1, nkb / 16);
    std::vector<int> c(nw, 1);
    if (nw < nsm) {
        double wsum = 0;
        for (auto& w : h.works) wsum += w.n + 3000.0;
        int used = 0;
        std::vector<std::pair<double, int>> frac;
        for (int i = 0; i < nw; ++i) {
            const double want = nsm * (h.works[i].n + 3000.0) / wsum;
            c[i] = std::max(1, (int)want);
            used += c[i];
            frac.push_back({want - (int)want, i});
        }
        std::sort(frac.begin(), frac.end(), [](auto& a, auto& b) { return a.first > b.first; });
        for (size_t k = 0; used < nsm && k < frac.size(); ++k, ++used) ++c[frac[k].second];
    }
    int cmax = 1;
    for (int i = 0; i < nw; ++i) {
        c[i] = std::min(c[i], maxc);
        cmax = std::max(cmax, c[i]);
    }
    h.lsup = (int)std::min<long long>(nkb, std::max(16 * cmax, 64));
    h.nsup = (int)((nkb + h.lsup - 1) / h.lsup);
    std::vector<int> first(nw);
    h.units.clear();
    for (int i = 0; i < nw; ++i) {
        first[i] = (int)h.units.size();
        for (int j = 0; j < c[i]; ++j) {
            const int a = (int)((long long)j * h.lsup / c[i]), b = (int)((long long)(j + 1) * h.lsup / c[i]);
            h.units.push_back(TcUnit{i, a, b - a, 0});
        }
    }
    for (BinLoc& L : h.loc) {
        const int w = L.work;
        L.work = first[w];
        L.pad = c[w];
    }
}

// Fields are numbered slot * pad + a (pad = nsh rounded up to 8) so that
// every box of 8 fields is one group of the K-block-major 16-bit planes.
TcSched build_tc_sched(const BinList& bins, const std::vector<int>& out_slots, int pad, size_t npts, int nsm,
                       int max_boxes = 12) {
    TcSched h;
    // a-range of each pair (b, c) over the bins, in groups of 8 shells
    std::map<std::pair<int, int>, std::pair<int, int>> arange;
    for (auto& t : bins) {
        auto it = arange.find({t[1], t[2]});
        if (it == arange.end()) arange[{t[1], t[2]}] = {t[0], t[0]};
        else it->second = {std::min(it->second.first, t[0]), std::max(it->second.second, t[0])};
    }
    // entries: a pair with a group range of at most 4 groups (a pair whose a-range is
    // longer appears once per piece), sorted by group range so that the 128 entries of
    // a tile need few groups: most tiles then fit one work of N <= 96 rows
    struct Entry { int glo, ghi, b, c; };
    std::vector<Entry> ent;
    for (auto& kv : arange) {
        int glo = kv.second.first / 8;
        const int ghi = kv.second.second / 8;
        while (ghi - glo + 1 > 4) {
            ent.push_back(Entry{glo, glo + 3, kv.first.first, kv.first.second});
            glo += 4;
        }
        ent.push_back(Entry{glo, ghi, kv.first.first, kv.first.second});
    }
    std::sort(ent.begin(), ent.end(), [](const Entry& x, const Entry& y) {
        return std::make_tuple(x.glo, x.ghi, x.b, x.c) < std::make_tuple(y.glo, y.ghi, y.b, y.c);
    });
    // per entry: (tile first work, tile first group, groups per slot, tile first entry, boxes per work)
    struct TileRef { int work0, g0, nbs, e0, per; };
    std::vector<TileRef> ref(ent.size());
    size_t i = 0;
    while (i < ent.size()) {
        int slo = ent[i].c, shi = ent[i].b, glo = ent[i].glo, ghi = ent[i].ghi;
        size_t j = i + 1;
        while (j < ent.size() && (int)(j - i) < 128) {
            const int nslo = std::min(slo, ent[j].c), nshi = std::max(shi, ent[j].b);
            if (nshi - nslo + 1 > 64) break;
            slo = nslo; shi = nshi;
            glo = std::min(glo, ent[j].glo); ghi = std::max(ghi, ent[j].ghi);
            ++j;
        }
        const int nbs = ghi - glo + 1;
        std::vector<int> boxes;
        for (int si : out_slots)
            for (int g = 0; g < nbs; ++g) boxes.push_back(si * pad + 8 * (glo + g));
        // works of at most max_boxes boxes (N <= 8 max_boxes, <= 96), split evenly
        const int work0 = (int)h.works.size();
        const int nwk = ((int)boxes.size() + max_boxes - 1) / max_boxes;
        const int per = ((int)boxes.size() + nwk - 1) / nwk;
        for (size_t b0 = 0; b0 < boxes.size(); b0 += per) {
            TcWork w{};
            w.pair0 = (int)i;
            w.npairs = (int)(j - i);
            w.shell_lo = slo;
            w.nshell = shi - slo + 1;
            w.nbox = (int)std::min<size_t>(per, boxes.size() - b0);
            w.n = (8 * w.nbox + 15) / 16 * 16;
            for (int b = 0; b < w.nbox; ++b) w.box_field[b] = boxes[b0 + b];
            h.works.push_back(w);
        }
        for (size_t e = i; e < j; ++e) ref[e] = TileRef{work0, glo, nbs, (int)i, per};
        i = j;
    }
    std::map<std::pair<int, int>, std::vector<int>> entries_of;   // pair -> its entries
    for (size_t e = 0; e < ent.size(); ++e) {
        h.pairs.push_back(int2{ent[e].b, ent[e].c});
        entries_of[{ent[e].b, ent[e].c}].push_back((int)e);
    }
    h.loc.resize(out_slots.size() * bins.size());
    for (size_t b = 0; b < bins.size(); ++b) {
        const int a = bins[b][0], ga = a / 8;
        int e = -1;
        for (int x : entries_of[{bins[b][1], bins[b][2]}])
            if (ent[x].glo <= ga && ga <= ent[x].ghi) e = x;
        const TileRef& t = ref[e];
        for (size_t si = 0; si < out_slots.size(); ++si) {
            const int box = (int)si * t.nbs + (ga - t.g0);
            // tensor-core slots are [field column][pair]: "row" holds the column
            h.loc[si * bins.size() + b] = BinLoc{t.work0 + box / t.per, 8 * (box % t.per) + a % 8, e - t.e0, 0};
        }
    }
    assign_units(h, npts, nsm);
    return h;
}

constexpr size_t TC_UNIT = 128 * 128;   // FP64 partial values per tensor-core CTA

}  // namespace

struct bsp_plan {
    int n = 0;
    double box = 0;
    int nsh = 0;
    std::vector<double> edges;
    std::vector<int> ells;       // output multipoles
    std::vector<int> slot_ell;   // field slots: slot 0 is l = 0
    std::vector<int> out_slots;  // slot of each output multipole
    int prec = 0;
    FftGeom geom{};
    int target_ctas = 2048;
    int fb_cap = 1;                   // FFT batch width the workspace was sized for
    int16_t* d_shell_of = nullptr;
    FieldDesc* d_fd_raw = nullptr;    // one field: delta on every mode but the mean (skew spectrum)
    int n2top = 0;                    // largest |n|^2 in a shell
    int ib_m = 0;                     // integrated bispectrum: cubes per side of the cached shell table
    int ib_n2top = 0;                 // largest |n_s|^2 of the sub-cube grid in a shell
    int16_t* d_shell_sub = nullptr;   // shell of each |n_s|^2 of the sub-cube grid (|n| = m |n_s|)
    cx<float>* d_tw32 = nullptr;
    cx<double>* d_tw64 = nullptr;
    FieldDesc* d_fd_delta = nullptr;  // [nslot*nsh], or [3][nslot*nsh] with shot noise
    bool shot = false;                // BSP_SHOT_NOISE: workspace for the shot-noise fields
    bool full = false;                // BSP_FULL_TENSOR: the Legendre leg on every shell of a bin
    // modal plans (Sec. 3.5): fields M^l_p from radial tables, all (a; b >= c) sums
    bool modal = false;
    int slot2 = -1;                   // slot of l = 2 (the U term of l = 4), or -1
    bool need_u = false;
    float* d_radial = nullptr;        // [n_funcs][n2max + 1]
    int* d_ells = nullptr;
    HostSched u_sched;                // rows M0_a, pairs M2_b M2_c
    DevSched u_dev;
    TcSched tc_u_sched;
    TcWork* d_tcu_works = nullptr;
    int2* d_tcu_pairs = nullptr;
    BinLoc* d_tcu_loc = nullptr;
    size_t upart_bytes = 0, tcu_part_bytes = 0, tfull_bytes = 0, ufull_bytes = 0;
    FieldDesc* d_fd_unit = nullptr;   // [nsh]
    // candidate bins (superset of the valid ones) and their counting schedule
    BinList cand;
    HostSched cand_sched;
    DevSched cand_dev;
    // counts on the fundamental domain of the cubic group: representative
    // points (linear index) and their orbit sizes
    uint32_t* d_rep_idx = nullptr;
    double* d_rep_w = nullptr;
    size_t nrep = 0;
    // valid bins after counts
    bool have_counts = false;
    BinList bins;                     // output bins (a; b >= c), the Legendre leg a
    std::vector<double> counts;
    BinList vbins;                    // valid sorted bins a >= b >= c and their counts
    std::vector<double> vcounts;
    double* d_counts = nullptr;
    HostSched comp_sched;
    DevSched comp_dev;
    // tensor-core path
    bool tc = false;
    int nprod = 3;
    FieldDesc* d_fd_tc = nullptr;     // [nslot*nsh]
    TcSched tc_sched;
    int nsm = 148;
    TcUnit* d_tc_units = nullptr;
    TcUnit* d_tcu_units = nullptr;
    TcWork* d_tc_works = nullptr;
    int2* d_tc_pairs = nullptr;
    BinLoc* d_tc_loc = nullptr;
    int* d_err = nullptr;
    unsigned* d_fmax = nullptr;   // per-field magnitude bounds for the 16-bit scaling
    int chunk_kb = 1;             // K-blocks (64 points each) per FP32 tensor-memory accumulation
    long long wait_cycles = 0;    // tensor-core pipeline wait limit in clock cycles (0: the kernel's default)
    int tc_max_boxes = 12;        // tensor-core works: at most this many boxes of 8 field rows (N <= 8 x this)
    size_t f0_bytes = 0, plane_bytes = 0, tc_part_bytes = 0;
    // workspace layout
    size_t fld32_bytes = 0, fld64_bytes = 0, t12_bytes32 = 0, t12_bytes64 = 0;
    int fb32 = 1, fb64 = 1;
    size_t part_bytes = 0, tout_bytes = 0, cnt_out_bytes = 0;
    size_t ws_bytes = 0, staging_bytes = 0;
    // optional per-phase CUDA-event timing of bsp_compute
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;      // 4 events per profiled call
    size_t ev_used = 0;
    int launches_last = 0;

    ~bsp_plan() {
        for (auto e : ev_pool) cudaEventDestroy(e);
        cudaFree(d_shell_of); cudaFree(d_tw32); cudaFree(d_tw64); cudaFree(d_fd_raw); cudaFree(d_shell_sub);
        cudaFree(d_fd_delta); cudaFree(d_fd_unit); cudaFree(d_counts);
        cudaFree(d_rep_idx); cudaFree(d_rep_w);
        cudaFree(d_fd_tc); cudaFree(d_tc_works); cudaFree(d_tc_pairs); cudaFree(d_tc_loc); cudaFree(d_err);
        cudaFree(d_fmax);
        cudaFree(d_tc_units); cudaFree(d_tcu_units);
        cudaFree(d_radial); cudaFree(d_ells); cudaFree(d_tcu_works); cudaFree(d_tcu_pairs); cudaFree(d_tcu_loc);
        u_dev.release();
        cand_dev.release(); comp_dev.release();
    }
    size_t npts() const { return (size_t)n * n * n; }
    size_t nkb() const { return (npts() + 63) / 64; }   // K-blocks of 64 points
    // tensor-core operands (K-block-major): F0 rows per K-block; 16-bit fields are
    // numbered slot * pad16 + a and stored in groups16 groups of 8 per K-block
    int kb_rows32 = 0, pad16 = 0, groups16 = 0;
    int nslot() const { return (int)slot_ell.size(); }
};

namespace {

void t12_sizes(const FftGeom& g, size_t elem, size_t* t1, size_t* t2) {
    *t1 = round256((size_t)g.nK * g.n * g.nKz * 2 * elem);
    *t2 = round256((size_t)g.n * g.n * g.nKz * 2 * elem);
}

// Offsets inside the workspace (the same for counts and compute; the two
// phases reuse the same bytes).
struct Layout {
    size_t fields, t1, t2, partial, tout, cnt, end;
};

Layout layout_compute(const bsp_plan* p) {
    Layout L{};
    size_t t1, t2;
    t12_sizes(p->geom, sizeof(float), &t1, &t2);
    L.fields = 0;
    if (p->tc) {
        // F0 (FP32 pair factors) | hi planes | lo planes (16-bit, nslot*nsh fields each)
        L.t1 = L.fields + p->f0_bytes + 2 * p->plane_bytes;
        L.t2 = L.t1 + t1 * p->fb32;
        L.partial = L.t2 + t2 * p->fb32;
        L.tout = L.partial + p->tc_part_bytes + p->tcu_part_bytes;
        L.cnt = L.tout + p->tout_bytes + p->tfull_bytes + p->ufull_bytes;
        L.end = L.cnt;
        return L;
    }
    if (p->modal) {
        L.t1 = L.fields + p->fld32_bytes;
        L.t2 = L.t1 + t1 * p->fb32;
        L.partial = L.t2 + t2 * p->fb32;
        L.tout = L.partial + p->part_bytes + p->upart_bytes;
        L.cnt = L.tout + p->tfull_bytes + p->ufull_bytes;
        L.end = L.cnt;
        return L;
    }
    L.t1 = L.fields + p->fld32_bytes;
    L.t2 = L.t1 + t1 * p->fb32;
    L.partial = L.t2 + t2 * p->fb32;
    L.tout = L.partial + p->part_bytes;
    L.cnt = L.tout + p->tout_bytes;
    L.end = L.cnt;
    return L;
}

Layout layout_counts(const bsp_plan* p) {
    Layout L{};
    size_t t1, t2;
    t12_sizes(p->geom, sizeof(double), &t1, &t2);
    L.fields = 0;
    L.t1 = L.fields + p->fld64_bytes;
    L.t2 = L.t1 + t1 * p->fb64;
    // the unit fields gathered on the representative points, weighted and
    // unweighted ([n_shells][nrep] FP64 each), then the partial sums
    L.partial = L.t2 + t2 * p->fb64 + 2 * round256((size_t)p->nsh * p->nrep * sizeof(double));
    L.tout = L.partial + round256(partial_bytes(p->cand_sched, CCOLS));
    L.cnt = L.tout;
    L.end = L.cnt + p->cnt_out_bytes;
    return L;
}

// Representatives of the orbits of the cubic group (axis permutations and
// sign flips, x -> n - x per axis) on the n^3 grid: 0 <= x <= y <= z <= n/2,
// with the orbit size (distinct permutations of (x, y, z) times 2 for every
// coordinate other than 0 and n/2).  A shell's unit field I_a(x) =
// sum_{m in a} cos(2 pi m.x / n) is invariant under the group (the shell
// depends on |m|^2 only), so sum_x I_a I_b I_c = sum_reps w I_a I_b I_c.
void cubic_reps(int n, std::vector<uint32_t>& idx, std::vector<double>& w) {
    const int h = n / 2;
    idx.clear();
    w.clear();
    for (int x = 0; x <= h; ++x)
        for (int y = x; y <= h; ++y)
            for (int z = y; z <= h; ++z) {
                const int perms = (x == y && y == z) ? 1 : (x == y || y == z) ? 3 : 6;
                int flips = 1;
                for (int v : {x, y, z})
                    if (v != 0 && v != h) flips *= 2;
                idx.push_back((uint32_t)(((size_t)x * n + y) * n + z));
                w.push_back((double)(perms * flips));
            }
}

bool good_size(int n) {
    if (n < 8 || n > 512 || n % 2) return false;
    int m = n;
    for (int q : {2, 3, 5})
        while (m % q == 0) m /= q;
    return m == 1;
}

}  // namespace

extern "C" {

const char* bsp_status_string(int s) {
    switch (s) {
        case BSP_OK: return "ok";
        case BSP_EINVAL: return "invalid argument";
        case BSP_ENOMEM: return "out of memory";
        case BSP_ECUDA: return "CUDA error";
        case BSP_EUNSUPPORTED: return "unsupported";
        case BSP_ETIMEOUT: return "device wait timed out";
        case BSP_ESTATE: return "call out of order";
        default: return "unknown status";
    }
}

const char* bsp_last_error(void) { return g_last_error.c_str(); }

int bsp_version(void) { return 100; }

bsp_status bsp_plan_create(bsp_plan** out, int n, double box, int n_shells, const double* edges_kf,
                           int n_ell, const int* ells, int prec, unsigned flags) {
    if (!out) return BSP_EINVAL;
    *out = nullptr;
    if (!good_size(n) || !(box > 0) || !std::isfinite(box) || n_shells < 1 || n_shells > 64 || !edges_kf ||
        n_ell < 1 || n_ell > 3 || !ells || (flags & ~(unsigned)(BSP_SHOT_NOISE | BSP_FULL_TENSOR)))
        return BSP_EINVAL;
    for (int i = 0; i <= n_shells; ++i)
        if (!(edges_kf[i] > 0) || !std::isfinite(edges_kf[i]) || (i && !(edges_kf[i] > edges_kf[i - 1])))
            return BSP_EINVAL;
    if (edges_kf[n_shells] > std::sqrt(3.0) * n / 2 + 1e-9) return BSP_EINVAL;
    for (int i = 0; i < n_ell; ++i) {
        if (ells[i] != 0 && ells[i] != 2 && ells[i] != 4) return BSP_EINVAL;
        if (i && ells[i] <= ells[i - 1]) return BSP_EINVAL;
    }
    if (prec != BSP_FP32 && prec != BSP_SPLIT_BF16 && prec != BSP_BF16 && prec != BSP_SPLIT_F16)
        return BSP_EUNSUPPORTED;
    if ((flags & BSP_SHOT_NOISE) && prec != BSP_FP32) return BSP_EUNSUPPORTED;

    bsp_plan* p = new (std::nothrow) bsp_plan();
    if (!p) return BSP_ENOMEM;
    p->n = n;
    p->box = box;
    p->nsh = n_shells;
    p->edges.assign(edges_kf, edges_kf + n_shells + 1);
    p->ells.assign(ells, ells + n_ell);
    p->prec = prec;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            p->nsm = sms;
    }
    p->shot = (flags & BSP_SHOT_NOISE) != 0;
    p->full = (flags & BSP_FULL_TENSOR) != 0;
    p->tc = prec != BSP_FP32;
    p->nprod = prec == BSP_BF16 ? 1 : 3;
    p->slot_ell.push_back(0);
    for (int l : p->ells)
        if (l != 0) p->slot_ell.push_back(l);
    for (int l : p->ells)
        for (int s = 0; s < p->nslot(); ++s)
            if (p->slot_ell[s] == l) p->out_slots.push_back(s);

    // geometry and pruning
    FftGeom& g = p->geom;
    g.n = n;
    const double emax = p->edges.back();
    int K = 0;
    while ((double)(K + 1) * (K + 1) < emax * emax) ++K;
    if (K >= n / 2) {
        g.K = n / 2; g.nK = n; g.pruned = 0; g.nKz = n / 2 + 1;
    } else {
        g.K = K; g.nK = 2 * K + 1; g.pruned = 1; g.nKz = K + 1;
    }
    g.n2max = 3 * (n / 2) * (n / 2);
    if (!radix_plan(n, g.rad, &g.nrad) || !radix_plan(n / 2, g.rad_h, &g.nrad_h)) {
        delete p;
        return BSP_EUNSUPPORTED;
    }

    // shell lookup by integer |n|^2: lo*lo <= n2 < hi*hi
    std::vector<int16_t> shell_of(g.n2max + 1, -1);
    for (int n2 = 0; n2 <= g.n2max; ++n2)
        for (int s = 0; s < n_shells; ++s) {
            double lo = p->edges[s], hi = p->edges[s + 1];
            if ((double)n2 >= lo * lo && (double)n2 < hi * hi) { shell_of[n2] = (int16_t)s; break; }
        }
    for (int n2 = 0; n2 <= g.n2max; ++n2)
        if (shell_of[n2] >= 0) p->n2top = n2;
    // per shell: the largest |frequency component| of its modes, floor(sqrt(max |n|^2))
    std::vector<int> kext(n_shells, 1);
    for (int n2 = 0, f = 0; n2 <= g.n2max; ++n2) {
        while ((long long)(f + 1) * (f + 1) <= n2) ++f;
        if (shell_of[n2] >= 0) kext[shell_of[n2]] = std::min(std::max(kext[shell_of[n2]], f), g.K);
    }
    std::vector<cx<double>> tw64(n);
    std::vector<cx<float>> tw32(n);
    for (int t = 0; t < n; ++t) {
        double ang = 2.0 * M_PI * (double)t / (double)n;
        tw64[t] = {std::cos(ang), std::sin(ang)};
        tw32[t] = {(float)tw64[t].re, (float)tw64[t].im};
    }
    std::vector<FieldDesc> fdd, fdu;
    std::vector<FieldDesc> fdt;
    const int pad16 = (n_shells + 7) & ~7;
    p->pad16 = pad16;
    p->groups16 = p->nslot() * pad16 / 8;
    for (int s = 0; s < p->nslot(); ++s)
        for (int a = 0; a < n_shells; ++a) {
            const int f = s * n_shells + a;
            fdd.push_back(FieldDesc{a, p->slot_ell[s], FIELD_DELTA, f, -1, kext[a], {0, 0}});
            fdt.push_back(FieldDesc{a, p->slot_ell[s], FIELD_DELTA, s == 0 ? a : -1, s * pad16 + a, kext[a], {0, 0}});
        }
    if (p->shot) {
        // S^l_a = w_l |delta|^2 on a, then W^l_a = w_l on a (W^0 = the unit fields I)
        const int nfs = p->nslot() * n_shells;
        for (int kind = 0; kind < 2; ++kind)
            for (int s = 0; s < p->nslot(); ++s)
                for (int a = 0; a < n_shells; ++a)
                    fdd.push_back(FieldDesc{a, p->slot_ell[s], kind == 0 ? FIELD_POWER : FIELD_UNIT,
                                            (kind + 1) * nfs + s * n_shells + a, -1, kext[a], {0, 0}});
    }
    for (int a = 0; a < n_shells; ++a) fdu.push_back(FieldDesc{a, 0, FIELD_UNIT, a, -1, kext[a], {0, 0}});
    bsp_status st;
    if ((st = upload(&p->d_shell_of, shell_of)) != BSP_OK || (st = upload(&p->d_tw32, tw32)) != BSP_OK ||
        (st = upload(&p->d_tw64, tw64)) != BSP_OK || (st = upload(&p->d_fd_delta, fdd)) != BSP_OK ||
        (st = upload(&p->d_fd_unit, fdu)) != BSP_OK || (st = upload(&p->d_fd_tc, fdt)) != BSP_OK ||
        (st = upload(&p->d_fd_raw, std::vector<FieldDesc>{FieldDesc{0, 0, FIELD_RAW, 0, -1, 0, {0, 0}}})) != BSP_OK ||
        (st = upload(&p->d_err, std::vector<int>{0, 0, 0})) != BSP_OK ||
        (st = upload(&p->d_fmax, std::vector<unsigned>((size_t)p->nslot() * pad16 + n_shells, 0u))) != BSP_OK) {
        delete p;
        return st;
    }

    // candidate bins: every (a >= b >= c) that can hold a triangle, either
    // without wrap-around (lo_a < hi_b + hi_c) or with it (hi_a+hi_b+hi_c > n)
    for (int a = 0; a < n_shells; ++a)
        for (int b = 0; b <= a; ++b)
            for (int c = 0; c <= b; ++c) {
                const double* e = p->edges.data();
                if (e[a] < e[b + 1] + e[c + 1] || e[a + 1] + e[b + 1] + e[c + 1] > n)
                    p->cand.push_back({a, b, c});
            }
    {
        std::vector<uint32_t> ridx;
        std::vector<double> rw;
        cubic_reps(n, ridx, rw);
        p->nrep = ridx.size();
        if ((st = upload(&p->d_rep_idx, ridx)) != BSP_OK || (st = upload(&p->d_rep_w, rw)) != BSP_OK) {
            delete p;
            return st;
        }
    }
    p->cand_sched = build_sched(p->cand, std::vector<int>{0}, n_shells, p->nrep, p->target_ctas, CCOLS);
    if ((st = upload_sched(p->cand_dev, p->cand_sched)) != BSP_OK) {
        delete p;
        return st;
    }
    // workspace sizing: compute schedule bounded by the candidate output bins
    const BinList ocand = p->full ? expand_full(p->cand) : p->cand;
    HostSched bound = build_sched(ocand, p->out_slots, n_shells, p->npts(), p->target_ctas, CCOLS);
    size_t t1, t2;
    t12_sizes(g, sizeof(float), &t1, &t2);
    const size_t nfields32 = (size_t)p->nslot() * n_shells;
    p->fld32_bytes = round256((p->shot ? 3 : 1) * nfields32 * p->npts() * sizeof(float));
    p->fb32 = (int)std::max<size_t>(1, std::min<size_t>(nfields32, (size_t)(2ull << 30) / (t1 + t2)));
    p->fb_cap = p->fb32;
    t12_sizes(g, sizeof(double), &t1, &t2);
    p->fld64_bytes = round256((size_t)n_shells * p->npts() * sizeof(double));
    p->fb64 = (int)std::max<size_t>(1, std::min<size_t>(n_shells, (size_t)(2ull << 30) / (t1 + t2)));
    // the valid-bin schedule has at most as many works as the bound, and
    // nsplit <= ceil(target / nwork), so nwork * nsplit <= target + nwork
    p->part_bytes = round256(std::max(partial_bytes(bound, CCOLS),
                                      (size_t)(4096 + bound.works.size()) * 64 * CCOLS * sizeof(double)));
    if (p->shot) p->part_bytes *= 4;   // main sum + three shot-noise sums
    p->tout_bytes = round256(p->ells.size() * ocand.size() * sizeof(double));
    if (p->tc) {
        p->kb_rows32 = n_shells;
        p->f0_bytes = round256((size_t)n_shells * p->nkb() * 256);
        p->plane_bytes = round256((size_t)p->groups16 * p->nkb() * 1024);   // hi and lo: 2 * plane_bytes
        // partial slots for the most works any tuning can make (works of 4 boxes)
        TcSched tb = build_tc_sched(ocand, p->out_slots, pad16, p->npts(), p->nsm, 4);
        p->tc_part_bytes = round256(std::max<size_t>((size_t)p->nsm, tb.units.size()) * TC_UNIT * sizeof(double));
    }
    p->cnt_out_bytes = round256(p->cand.size() * sizeof(double));
    p->ws_bytes = std::max(layout_compute(p).end, layout_counts(p).end);
    p->staging_bytes = round256((size_t)n * n * (n / 2 + 1) * 8) + p->tout_bytes;
    *out = p;
    return BSP_OK;
}

bsp_status bsp_plan_create_modal(bsp_plan** out, int n, double box, int n_funcs, const double* radial, int n_ell,
                                 const int* ells, int prec, unsigned flags) {
    if (!out) return BSP_EINVAL;
    *out = nullptr;
    if (!good_size(n) || !(box > 0) || !std::isfinite(box) || n_funcs < 1 || n_funcs > 64 || !radial ||
        n_ell < 1 || n_ell > 3 || !ells || flags != 0)
        return BSP_EINVAL;
    for (int i = 0; i < n_ell; ++i) {
        if (ells[i] != 0 && ells[i] != 2 && ells[i] != 4) return BSP_EINVAL;
        if (i && ells[i] <= ells[i - 1]) return BSP_EINVAL;
    }
    if (prec != BSP_FP32 && prec != BSP_SPLIT_BF16 && prec != BSP_BF16 && prec != BSP_SPLIT_F16)
        return BSP_EUNSUPPORTED;
    const int n2max = 3 * (n / 2) * (n / 2);
    std::vector<float> tab((size_t)n_funcs * (n2max + 1));
    int maxn2 = 0;
    for (int f = 0; f < n_funcs; ++f)
        for (int n2 = 0; n2 <= n2max; ++n2) {
            const double v = radial[(size_t)f * (n2max + 1) + n2];
            if (!std::isfinite(v)) return BSP_EINVAL;
            tab[(size_t)f * (n2max + 1) + n2] = (float)v;
            if (v != 0.0 && n2 > maxn2) maxn2 = n2;
        }
    if (maxn2 == 0) return BSP_EINVAL;

    bsp_plan* p = new (std::nothrow) bsp_plan();
    if (!p) return BSP_ENOMEM;
    p->modal = true;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            p->nsm = sms;
    }
    p->n = n;
    p->box = box;
    p->nsh = n_funcs;
    p->ells.assign(ells, ells + n_ell);
    p->prec = prec;
    p->tc = prec != BSP_FP32;
    p->nprod = prec == BSP_BF16 ? 1 : 3;
    p->slot_ell.push_back(0);
    for (int l : p->ells)
        if (l != 0) p->slot_ell.push_back(l);
    for (int l : p->ells)
        for (int s = 0; s < p->nslot(); ++s)
            if (p->slot_ell[s] == l) p->out_slots.push_back(s);
    for (int s = 0; s < p->nslot(); ++s)
        if (p->slot_ell[s] == 2) p->slot2 = s;
    for (int l : p->ells)
        if (l == 4) p->need_u = true;
    if (p->need_u && p->slot2 < 0) {
        // the l = 4 sum needs the l = 2 fields even when l = 2 is not an output
        p->slot_ell.push_back(2);
        p->slot2 = p->nslot() - 1;
    }
    FftGeom& g = p->geom;
    g.n = n;
    int K = 0;
    while ((K + 1) * (K + 1) <= maxn2) ++K;
    if (K >= n / 2) {
        g.K = n / 2; g.nK = n; g.pruned = 0; g.nKz = n / 2 + 1;
    } else {
        g.K = K; g.nK = 2 * K + 1; g.pruned = 1; g.nKz = K + 1;
    }
    g.n2max = n2max;
    if (!radix_plan(n, g.rad, &g.nrad) || !radix_plan(n / 2, g.rad_h, &g.nrad_h)) {
        delete p;
        return BSP_EUNSUPPORTED;
    }
    std::vector<cx<double>> tw64(n);
    std::vector<cx<float>> tw32(n);
    for (int t = 0; t < n; ++t) {
        const double ang = 2.0 * M_PI * (double)t / (double)n;
        tw64[t] = {std::cos(ang), std::sin(ang)};
        tw32[t] = {(float)tw64[t].re, (float)tw64[t].im};
    }
    // fields M^l_a = sum w_l R_a[n^2] delta e^{ik.x}; on the tensor-core path the
    // FP32 copies are the pair factors: slot 0, then slot2 (for U) at index nf + a
    const int nf = n_funcs;
    std::vector<FieldDesc> fdd, fdt;
    p->pad16 = (nf + 7) & ~7;
    p->groups16 = p->nslot() * p->pad16 / 8;
    for (int s = 0; s < p->nslot(); ++s)
        for (int a = 0; a < nf; ++a) {
            const int f = s * nf + a;
            fdd.push_back(FieldDesc{a, p->slot_ell[s], FIELD_RADIAL, f, -1, 0, {0, 0}});
            int o32 = -1;
            if (s == 0) o32 = a;
            else if (p->need_u && s == p->slot2) o32 = nf + a;
            fdt.push_back(FieldDesc{a, p->slot_ell[s], FIELD_RADIAL, o32, s * p->pad16 + a, 0, {0, 0}});
        }
    bsp_status st;
    if ((st = upload(&p->d_radial, tab)) != BSP_OK || (st = upload(&p->d_tw32, tw32)) != BSP_OK ||
        (st = upload(&p->d_tw64, tw64)) != BSP_OK || (st = upload(&p->d_fd_delta, fdd)) != BSP_OK ||
        (st = upload(&p->d_fd_tc, fdt)) != BSP_OK || (st = upload(&p->d_err, std::vector<int>{0, 0, 0})) != BSP_OK ||
        (st = upload(&p->d_ells, p->ells)) != BSP_OK ||
        (st = upload(&p->d_fmax, std::vector<unsigned>((size_t)p->nslot() * p->pad16 + 2 * nf, 0u))) != BSP_OK) {
        delete p;
        return st;
    }
    // every (a; b >= c): T^l for all slots, U on slot 0 rows
    for (int a = 0; a < nf; ++a)
        for (int b = 0; b < nf; ++b)
            for (int c = 0; c <= b; ++c) p->bins.push_back({a, b, c});
    p->counts.assign(p->bins.size(), 1.0);
    const size_t nall = p->bins.size();
    size_t t1, t2;
    t12_sizes(g, sizeof(float), &t1, &t2);
    const size_t nfields = (size_t)p->nslot() * nf;
    p->fb32 = (int)std::max<size_t>(1, std::min<size_t>(nfields, (size_t)(2ull << 30) / (t1 + t2)));
    p->tfull_bytes = round256(p->ells.size() * nall * sizeof(double));
    p->ufull_bytes = p->need_u ? round256(nall * sizeof(double)) : 0;
    if (!p->tc) {
        p->comp_sched = build_sched(p->bins, p->out_slots, nf, p->npts(), p->target_ctas, CCOLS);
        p->fld32_bytes = round256(nfields * p->npts() * sizeof(float));
        p->part_bytes = round256(partial_bytes(p->comp_sched, CCOLS));
        if ((st = upload_sched(p->comp_dev, p->comp_sched)) != BSP_OK) {
            delete p;
            return st;
        }
        if (p->need_u) {
            p->u_sched = build_sched(p->bins, std::vector<int>{0}, nf, p->npts(), p->target_ctas, CCOLS);
            p->upart_bytes = round256(partial_bytes(p->u_sched, CCOLS));
            if ((st = upload_sched(p->u_dev, p->u_sched)) != BSP_OK) {
                delete p;
                return st;
            }
        }
    } else {
        p->tc_sched = build_tc_sched(p->bins, p->out_slots, p->pad16, p->npts(), p->nsm);
        p->kb_rows32 = (p->need_u ? 2 : 1) * nf;
        p->f0_bytes = round256((size_t)p->kb_rows32 * p->nkb() * 256);
        p->plane_bytes = round256((size_t)p->groups16 * p->nkb() * 1024);   // hi and lo: 2 * plane_bytes
        p->tc_part_bytes = round256(p->tc_sched.units.size() * TC_UNIT * sizeof(double));
        if ((st = upload(&p->d_tc_units, p->tc_sched.units)) != BSP_OK ||
            (st = upload(&p->d_tc_works, p->tc_sched.works)) != BSP_OK ||
            (st = upload(&p->d_tc_pairs, p->tc_sched.pairs)) != BSP_OK ||
            (st = upload(&p->d_tc_loc, p->tc_sched.loc)) != BSP_OK) {
            delete p;
            return st;
        }
        if (p->need_u) {
            p->tc_u_sched = build_tc_sched(p->bins, std::vector<int>{0}, p->pad16, p->npts(), p->nsm);
            p->tcu_part_bytes = round256(p->tc_u_sched.units.size() * TC_UNIT * sizeof(double));
            if ((st = upload(&p->d_tcu_units, p->tc_u_sched.units)) != BSP_OK ||
                (st = upload(&p->d_tcu_works, p->tc_u_sched.works)) != BSP_OK ||
                (st = upload(&p->d_tcu_pairs, p->tc_u_sched.pairs)) != BSP_OK ||
                (st = upload(&p->d_tcu_loc, p->tc_u_sched.loc)) != BSP_OK) {
                delete p;
                return st;
            }
        }
    }
    if ((st = upload(&p->d_counts, p->counts)) != BSP_OK) {
        delete p;
        return st;
    }
    p->have_counts = true;
    p->ws_bytes = layout_compute(p).end;
    p->staging_bytes = 0;
    *out = p;
    return BSP_OK;
}

bsp_status bsp_modal_size(const bsp_plan* p, int* n_funcs, int* n_trip) {
    if (!p || !p->modal) return BSP_EINVAL;
    const int nf = p->nsh;
    if (n_funcs) *n_funcs = nf;
    if (n_trip) *n_trip = nf * (nf + 1) * (nf + 2) / 6;
    return BSP_OK;
}

void bsp_plan_destroy(bsp_plan* p) { delete p; }

bsp_status bsp_workspace_size(const bsp_plan* p, size_t* bytes) {
    if (!p || !bytes) return BSP_EINVAL;
    *bytes = p->ws_bytes;
    return BSP_OK;
}

bsp_status bsp_host_staging_size(const bsp_plan* p, size_t* bytes) {
    if (!p || !bytes) return BSP_EINVAL;
    *bytes = p->staging_bytes;
    return BSP_OK;
}

// After the valid bins and counts are known: contraction schedules and the
// device copy of the counts.
// Output bins from the valid sorted bins: the sorted list itself, or with
// BSP_FULL_TENSOR every distinct (a; b >= c) whose shells are a valid sorted
// bin, lexicographic, each with that bin's count.
static void set_output_bins(bsp_plan* p) {
    if (!p->full) {
        p->bins = p->vbins;
        p->counts = p->vcounts;
        return;
    }
    std::map<std::array<int, 3>, double> cnt;   // sorted shells -> count
    for (size_t i = 0; i < p->vbins.size(); ++i) cnt[p->vbins[i]] = p->vcounts[i];
    p->bins = expand_full(p->vbins);
    p->counts.clear();
    for (const auto& t : p->bins) {
        std::array<int, 3> s = t;
        std::sort(s.begin(), s.end(), [](int x, int y) { return x > y; });
        p->counts.push_back(cnt[s]);
    }
}

static bsp_status finish_counts(bsp_plan* p) {
    p->comp_sched = build_sched(p->bins, p->out_slots, p->nsh, p->npts(), p->target_ctas, CCOLS);
    if (round256(partial_bytes(p->comp_sched, CCOLS)) * (p->shot ? 4 : 1) > p->part_bytes) return BSP_ENOMEM;
    bsp_status s = upload_sched(p->comp_dev, p->comp_sched);
    if (s != BSP_OK) return s;
    if (p->tc) {
        p->tc_sched = build_tc_sched(p->bins, p->out_slots, p->pad16, p->npts(), p->nsm, p->tc_max_boxes);
        if (round256(p->tc_sched.units.size() * TC_UNIT * sizeof(double)) > p->tc_part_bytes) return BSP_ENOMEM;
        cudaFree(p->d_tc_works); cudaFree(p->d_tc_pairs); cudaFree(p->d_tc_loc); cudaFree(p->d_tc_units);
        p->d_tc_works = nullptr; p->d_tc_pairs = nullptr; p->d_tc_loc = nullptr; p->d_tc_units = nullptr;
        if ((s = upload(&p->d_tc_units, p->tc_sched.units)) != BSP_OK) return s;
        if ((s = upload(&p->d_tc_works, p->tc_sched.works)) != BSP_OK) return s;
        if ((s = upload(&p->d_tc_pairs, p->tc_sched.pairs)) != BSP_OK) return s;
        if ((s = upload(&p->d_tc_loc, p->tc_sched.loc)) != BSP_OK) return s;
    }
    cudaFree(p->d_counts);
    p->d_counts = nullptr;
    if ((s = upload(&p->d_counts, p->counts)) != BSP_OK) return s;
    p->have_counts = true;
    return BSP_OK;
}

bsp_status bsp_counts(bsp_plan* p, void* ws, void* stream) {
    if (!p || !ws || !aligned256(ws) || p->modal) return BSP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const Layout L = layout_counts(p);
    char* base = (char*)ws;
    double* f64 = (double*)(base + L.fields);
    cx<double>* t1 = (cx<double>*)(base + L.t1);
    cx<double>* t2 = (cx<double>*)(base + L.t2);
    size_t t1s, t2s;
    t12_sizes(p->geom, sizeof(double), &t1s, &t2s);
    // unit fields I_a (FP64), in batches of fb64 fields
    for (int f0 = 0; f0 < p->nsh; f0 += p->fb64) {
        int nf = std::min(p->fb64, p->nsh - f0);
        cudaError_t e = launch_fft_fields<double>(p->geom, nullptr, p->d_shell_of, nullptr, p->d_fd_unit + f0, nf,
                                                  p->d_tw64, t1, t2, f64, p->npts(), nullptr, nullptr, 0, nullptr,
                                                  nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "fft (counts)");
    }
    // gather the unit fields on the representatives of the cubic group's
    // orbits (weighted rows, unweighted pair factors), then contract there
    const size_t cbytes = round256((size_t)p->nsh * p->nrep * sizeof(double));
    double* wrows = (double*)(base + L.partial - 2 * cbytes);
    double* urows = (double*)(base + L.partial - cbytes);
    cudaError_t e = launch_gather_reps(f64, p->npts(), p->nsh, p->d_rep_idx, p->d_rep_w, p->nrep, wrows, urows, st);
    if (e != cudaSuccess) return cuda_fail(e, "gather (counts)");
    double* partial = (double*)(base + L.partial);
    double* cnt = (double*)(base + L.cnt);
    e = launch_contract_cc<double>(wrows, urows, nullptr, 0, p->nrep, p->cand_dev.works, p->cand_dev.nwork,
                                   p->cand_dev.pairs, p->cand_dev.rowf, p->nrep, p->cand_dev.nsplit, partial, st);
    if (e != cudaSuccess) return cuda_fail(e, "contract (counts)");
    const double n3 = (double)p->npts();
    e = launch_reduce(partial, p->cand_dev.nsplit, 0, 0, p->cand_dev.loc, (int)p->cand.size(),
                      (int)p->cand.size(), nullptr, 1.0 / n3, 0, nullptr, cnt, st);
    if (e != cudaSuccess) return cuda_fail(e, "reduce (counts)");
    std::vector<double> hc(p->cand.size());
    CK(cudaMemcpyAsync(hc.data(), cnt, sizeof(double) * hc.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    p->vbins.clear();
    p->vcounts.clear();
    for (size_t i = 0; i < p->cand.size(); ++i)
        if (hc[i] >= 1.0) {
            p->vbins.push_back(p->cand[i]);
            p->vcounts.push_back(hc[i]);
        }
    set_output_bins(p);
    return finish_counts(p);
}

bsp_status bsp_plan_share_counts(bsp_plan* dst, const bsp_plan* src) {
    if (!dst || !src || dst == src) return BSP_EINVAL;
    if (!src->have_counts) return BSP_ESTATE;
    if (dst->n != src->n || dst->nsh != src->nsh || dst->edges != src->edges) return BSP_EINVAL;
    dst->vbins = src->vbins;
    dst->vcounts = src->vcounts;
    set_output_bins(dst);
    return finish_counts(dst);
}

bsp_status bsp_plan_bins(const bsp_plan* p, int* n_bins, int32_t* abc, double* counts) {
    if (!p || !n_bins) return BSP_EINVAL;
    if (!p->have_counts) return BSP_ESTATE;
    *n_bins = (int)p->bins.size();
    for (size_t i = 0; i < p->bins.size(); ++i) {
        if (abc)
            for (int k = 0; k < 3; ++k) abc[3 * i + k] = p->bins[i][k];
        if (counts) counts[i] = p->counts[i];
    }
    return BSP_OK;
}

bsp_status bsp_bins_aliased(int n, int n_shells, const double* edges_kf, int n_bins, const int32_t* abc,
                            int32_t* flags) {
    if (n < 2 || n_shells < 1 || !edges_kf || n_bins < 0 || (n_bins && (!abc || !flags))) return BSP_EINVAL;
    for (int i = 0; i <= n_shells; ++i)
        if (!(edges_kf[i] > 0) || !std::isfinite(edges_kf[i]) || (i && !(edges_kf[i] > edges_kf[i - 1])))
            return BSP_EINVAL;
    for (int i = 0; i < 3 * n_bins; ++i)
        if (abc[i] < 0 || abc[i] >= n_shells) return BSP_EINVAL;
    // a mode of shell s has every component below hi_s in size, so q1 + q2 + q3
    // can only be a nonzero multiple of n when hi_a + hi_b + hi_c > n
    for (int i = 0; i < n_bins; ++i)
        flags[i] = edges_kf[abc[3 * i] + 1] + edges_kf[abc[3 * i + 1] + 1] + edges_kf[abc[3 * i + 2] + 1] > (double)n
                       ? 1 : 0;
    return BSP_OK;
}

static bsp_status mark(bsp_plan* p, cudaStream_t st, int k) {
    if (!p->profiling) return BSP_OK;
    size_t need = p->ev_used + 1;
    while (p->ev_pool.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        p->ev_pool.push_back(e);
    }
    (void)k;
    CK(cudaEventRecord(p->ev_pool[p->ev_used++], st));
    return BSP_OK;
}

// The last K-block of the tensor-core operands is partly past the grid when
// n^3 is not a multiple of 64: zero it before the FFT fills the rest.
static bsp_status clear_tail(bsp_plan* p, float* f0, uint32_t* planes, cudaStream_t st) {
    if (p->npts() % 64 == 0) return BSP_OK;
    const size_t kb = p->nkb() - 1;
    CK(cudaMemsetAsync((char*)f0 + kb * p->kb_rows32 * 256, 0, (size_t)p->kb_rows32 * 256, st));
    CK(cudaMemsetAsync((char*)planes + kb * p->groups16 * 2048, 0, (size_t)p->groups16 * 2048, st));
    return BSP_OK;
}

static bsp_status compute_impl(bsp_plan* p, const void* delta_k, double nbar, void* ws, cudaStream_t st,
                               double* B) {
    if (nbar != 0.0 && !p->shot) return p->tc ? BSP_EUNSUPPORTED : BSP_EINVAL;
    if (p->profiling && p->ev_used % 4 != 0) return BSP_ESTATE;
    bsp_status ms;
    if ((ms = mark(p, st, 0)) != BSP_OK) return ms;
    int launches = 0;
    const Layout L = layout_compute(p);
    char* base = (char*)ws;
    if (p->tc) {
        float* f0 = (float*)(base + L.fields);
        uint32_t* hi = (uint32_t*)(base + L.fields + p->f0_bytes);   // hi and lo, K-block-major groups
        cx<float>* t1 = (cx<float>*)(base + L.t1);
        cx<float>* t2 = (cx<float>*)(base + L.t2);
        const int nf = p->nslot() * p->nsh;
        unsigned* fmax2 = p->d_fmax;              // [slot * pad16 + a]  max |T2| per field (bounds |F|)
        CK(cudaMemsetAsync(p->d_fmax, 0, sizeof(unsigned) * ((size_t)p->nslot() * p->pad16 + p->nsh), st));
        CK(cudaMemsetAsync(p->d_err, 0, 3 * sizeof(int), st));   // error code
        if ((ms = clear_tail(p, f0, hi, st)) != BSP_OK) return ms;
        const int f16 = p->prec == BSP_SPLIT_F16 ? 1 : 0;
        for (int f0i = 0; f0i < nf; f0i += p->fb32) {
            int nb = std::min(p->fb32, nf - f0i);
            cudaError_t e = launch_fft_fields<float>(p->geom, (const cx<float>*)delta_k, p->d_shell_of, nullptr,
                                                     p->d_fd_tc + f0i, nb, p->d_tw32, t1, t2, f0, p->npts(), hi,
                                                     p->nprod == 3 ? hi : nullptr, f16, fmax2, nullptr, st,
                                                     FieldLayout{p->kb_rows32, p->groups16});
            if (e != cudaSuccess) return cuda_fail(e, "fft");
            launches += 3;
        }
        if ((ms = mark(p, st, 1)) != BSP_OK) return ms;
        double* partial = (double*)(base + L.partial);
        double* tout = (double*)(base + L.tout);
        CK(cudaMemsetAsync(partial, 0, p->tc_sched.units.size() * TC_UNIT * sizeof(double), st));
        cudaError_t e = launch_contract_tc(f16 != 0, f0, p->kb_rows32, 0, hi, p->groups16, (long long)p->nkb(),
                                           p->d_tc_works, p->d_tc_units,
                                           (int)p->tc_sched.units.size(), p->tc_sched.lsup, p->tc_sched.nsup,
                                           p->d_tc_pairs, 0, fmax2, 2.f * (float)p->geom.nKz, p->nprod,
                                           p->chunk_kb, partial, p->d_err, st, p->wait_cycles);
        if (e != cudaSuccess) return cuda_fail(e, "contract (tensor cores)");
        if ((ms = mark(p, st, 2)) != BSP_OK) return ms;
        const double V = p->box * p->box * p->box;
        e = launch_reduce(partial, 0, TC_UNIT, 128, p->d_tc_loc, (int)p->tc_sched.loc.size(),
                          (int)p->bins.size(), p->d_counts, 1.0 / (V * (double)p->npts()), 1, tout, B, st);
        if (e != cudaSuccess) return cuda_fail(e, "reduce");
        if ((ms = mark(p, st, 3)) != BSP_OK) return ms;
        p->launches_last = launches + 2;
        return BSP_OK;
    }
    float* f32 = (float*)(base + L.fields);
    cx<float>* t1 = (cx<float>*)(base + L.t1);
    cx<float>* t2 = (cx<float>*)(base + L.t2);
    const int nf = p->nslot() * p->nsh;
    const bool shot = nbar > 0.0;
    const int nft = shot ? 3 * nf : nf;   // F, then S and W with shot noise
    for (int f0 = 0; f0 < nft; f0 += p->fb32) {
        int nb = std::min(p->fb32, nft - f0);
        cudaError_t e = launch_fft_fields<float>(p->geom, (const cx<float>*)delta_k, p->d_shell_of, nullptr,
                                                 p->d_fd_delta + f0, nb, p->d_tw32, t1, t2, f32, p->npts(), nullptr,
                                                 nullptr, 0, nullptr, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "fft");
        launches += 3;
    }
    if ((ms = mark(p, st, 1)) != BSP_OK) return ms;
    double* partial = (double*)(base + L.partial);
    double* tout = (double*)(base + L.tout);
    const size_t pstride = round256(partial_bytes(p->comp_sched, CCOLS)) / sizeof(double);
    const size_t fs = (size_t)nf * p->npts();
    const float* F = f32;
    const float* S = f32 + fs;
    const float* W = f32 + 2 * fs;   // slot 0 of W: the unit fields I
    struct Job { const float *rows, *px, *py; int sym; };
    Job jobs[4] = {{F, F, nullptr, 0},      // T: rows F^l_a, pairs F_b F_c
                   {S, W, nullptr, 0},      // rows S^l_a (w_l |delta|^2), pairs I_b I_c
                   {W, S, W, 1},            // rows W^l_a, pairs S_b I_c + I_b S_c
                   {W, W, nullptr, 0}};     // rows W^l_a, pairs I_b I_c
    for (int j = 0; j < (shot ? 4 : 1); ++j) {
        cudaError_t e = launch_contract_cc<float>(jobs[j].rows, jobs[j].px, jobs[j].py, jobs[j].sym, p->npts(),
                                                  p->comp_dev.works, p->comp_dev.nwork, p->comp_dev.pairs,
                                                  p->comp_dev.rowf, p->npts(), p->comp_dev.nsplit,
                                                  partial + j * pstride, st);
        if (e != cudaSuccess) return cuda_fail(e, "contract");
        ++launches;
    }
    if ((ms = mark(p, st, 2)) != BSP_OK) return ms;
    const double V = p->box * p->box * p->box, n3 = (double)p->npts();
    // B = [T / V - (T_S + T_SI) / (V nbar) + 2 T_W / nbar^2] / (n^3 N_abc)   (Poisson shot noise)
    ShotTerms sh{};
    if (shot) {
        sh.n = 3;
        sh.partial[0] = partial + pstride;
        sh.partial[1] = partial + 2 * pstride;
        sh.partial[2] = partial + 3 * pstride;
        sh.coef[0] = 1.0 / (V * nbar * n3);
        sh.coef[1] = 1.0 / (V * nbar * n3);
        sh.coef[2] = -2.0 / (nbar * nbar * n3);
    }
    cudaError_t e = launch_reduce(partial, p->comp_dev.nsplit, 0, 0, p->comp_dev.loc, p->comp_dev.nloc,
                                  (int)p->bins.size(), p->d_counts, 1.0 / (V * n3), 1, tout, B, st,
                                  shot ? &sh : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "reduce");
    if ((ms = mark(p, st, 3)) != BSP_OK) return ms;
    p->launches_last = launches + 1;
    return BSP_OK;
}

bsp_status bsp_modal_compute(bsp_plan* p, const void* delta_k, void* ws, void* stream, double* S) {
    if (!p || !p->modal || !delta_k || !ws || !S || !aligned256(delta_k) || !aligned256(ws) || !aligned256(S))
        return BSP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const Layout L = layout_compute(p);
    char* base = (char*)ws;
    const int nf = p->nsh, nfields = p->nslot() * nf;
    const size_t nall = p->bins.size();
    const int ntrip = nf * (nf + 1) * (nf + 2) / 6;
    double* tfull = (double*)(base + L.tout);
    double* ufull = p->need_u ? (double*)(base + L.tout + p->tfull_bytes) : nullptr;
    const double V = p->box * p->box * p->box, n3 = (double)p->npts();
    bsp_status ms;
    if ((ms = mark(p, st, 0)) != BSP_OK) return ms;
    int launches = 0;
    if (!p->tc) {
        float* f32 = (float*)(base + L.fields);
        cx<float>* t1 = (cx<float>*)(base + L.t1);
        cx<float>* t2 = (cx<float>*)(base + L.t2);
        for (int f0 = 0; f0 < nfields; f0 += p->fb32) {
            const int nb = std::min(p->fb32, nfields - f0);
            cudaError_t e = launch_fft_fields<float>(p->geom, (const cx<float>*)delta_k, nullptr, p->d_radial,
                                                     p->d_fd_delta + f0, nb, p->d_tw32, t1, t2, f32, p->npts(),
                                                     nullptr, nullptr, 0, nullptr, nullptr, st);
            if (e != cudaSuccess) return cuda_fail(e, "fft (modal)");
            launches += 3;
        }
        if ((ms = mark(p, st, 1)) != BSP_OK) return ms;
        double* part = (double*)(base + L.partial);
        cudaError_t e = launch_contract_cc<float>(f32, f32, nullptr, 0, p->npts(), p->comp_dev.works,
                                                  p->comp_dev.nwork, p->comp_dev.pairs, p->comp_dev.rowf,
                                                  p->npts(), p->comp_dev.nsplit, part, st);
        if (e != cudaSuccess) return cuda_fail(e, "contract (modal)");
        ++launches;
        if (p->need_u) {
            const float* m2 = f32 + (size_t)p->slot2 * nf * p->npts();
            e = launch_contract_cc<float>(f32, m2, nullptr, 0, p->npts(), p->u_dev.works, p->u_dev.nwork,
                                          p->u_dev.pairs, p->u_dev.rowf, p->npts(), p->u_dev.nsplit,
                                          part + p->part_bytes / sizeof(double), st);
            if (e != cudaSuccess) return cuda_fail(e, "contract (modal U)");
            ++launches;
        }
        if ((ms = mark(p, st, 2)) != BSP_OK) return ms;
        e = launch_reduce(part, p->comp_dev.nsplit, 0, 0, p->comp_dev.loc, p->comp_dev.nloc, (int)nall,
                          p->d_counts, 1.0, 2, nullptr, tfull, st);
        if (e == cudaSuccess && p->need_u)
            e = launch_reduce(part + p->part_bytes / sizeof(double), p->u_dev.nsplit, 0, 0, p->u_dev.loc,
                              p->u_dev.nloc, (int)nall, p->d_counts, 1.0, 2, nullptr, ufull, st);
        if (e != cudaSuccess) return cuda_fail(e, "reduce (modal)");
        launches += p->need_u ? 2 : 1;
    } else {
        float* f0 = (float*)(base + L.fields);
        uint32_t* hi = (uint32_t*)(base + L.fields + p->f0_bytes);
        cx<float>* t1 = (cx<float>*)(base + L.t1);
        cx<float>* t2 = (cx<float>*)(base + L.t2);
        unsigned* fmax2 = p->d_fmax;                    // [slot * pad16 + a] max |T2| per field (bounds |F|)
        CK(cudaMemsetAsync(p->d_fmax, 0, sizeof(unsigned) * ((size_t)p->nslot() * p->pad16 + 2 * nf), st));
        CK(cudaMemsetAsync(p->d_err, 0, 3 * sizeof(int), st));   // error code
        if ((ms = clear_tail(p, f0, hi, st)) != BSP_OK) return ms;
        const int f16 = p->prec == BSP_SPLIT_F16 ? 1 : 0;
        for (int fi = 0; fi < nfields; fi += p->fb32) {
            const int nb = std::min(p->fb32, nfields - fi);
            cudaError_t e = launch_fft_fields<float>(p->geom, (const cx<float>*)delta_k, nullptr, p->d_radial,
                                                     p->d_fd_tc + fi, nb, p->d_tw32, t1, t2, f0, p->npts(), hi,
                                                     p->nprod == 3 ? hi : nullptr, f16, fmax2, nullptr, st,
                                                     FieldLayout{p->kb_rows32, p->groups16});
            if (e != cudaSuccess) return cuda_fail(e, "fft (modal)");
            launches += 3;
        }
        if ((ms = mark(p, st, 1)) != BSP_OK) return ms;
        double* part = (double*)(base + L.partial);
        double* upart = (double*)(base + L.partial + p->tc_part_bytes);
        CK(cudaMemsetAsync(part, 0, p->tc_sched.units.size() * TC_UNIT * sizeof(double), st));
        if (p->need_u) CK(cudaMemsetAsync(upart, 0, p->tc_u_sched.units.size() * TC_UNIT * sizeof(double), st));
        cudaError_t e = launch_contract_tc(f16 != 0, f0, p->kb_rows32, 0, hi, p->groups16, (long long)p->nkb(),
                                           p->d_tc_works, p->d_tc_units,
                                           (int)p->tc_sched.units.size(), p->tc_sched.lsup, p->tc_sched.nsup,
                                           p->d_tc_pairs, 0, fmax2, 2.f * (float)p->geom.nKz, p->nprod,
                                           p->chunk_kb, part, p->d_err, st, p->wait_cycles);
        if (e != cudaSuccess) return cuda_fail(e, "contract (modal, tensor cores)");
        ++launches;
        if (p->need_u) {
            e = launch_contract_tc(f16 != 0, f0, p->kb_rows32, nf, hi, p->groups16, (long long)p->nkb(),
                                   p->d_tcu_works, p->d_tcu_units,
                                   (int)p->tc_u_sched.units.size(), p->tc_u_sched.lsup, p->tc_u_sched.nsup,
                                   p->d_tcu_pairs, p->slot2 * p->pad16, fmax2, 2.f * (float)p->geom.nKz, p->nprod,
                                   p->chunk_kb, upart, p->d_err, st, p->wait_cycles);
            if (e != cudaSuccess) return cuda_fail(e, "contract (modal U, tensor cores)");
            ++launches;
        }
        if ((ms = mark(p, st, 2)) != BSP_OK) return ms;
        e = launch_reduce(part, 0, TC_UNIT, 128, p->d_tc_loc, (int)p->tc_sched.loc.size(),
                          (int)nall, p->d_counts, 1.0, 2, nullptr, tfull, st);
        if (e == cudaSuccess && p->need_u)
            e = launch_reduce(upart, 0, TC_UNIT, 128, p->d_tcu_loc,
                              (int)p->tc_u_sched.loc.size(), (int)nall, p->d_counts, 1.0, 2, nullptr, ufull, st);
        if (e != cudaSuccess) return cuda_fail(e, "reduce (modal)");
        launches += p->need_u ? 2 : 1;
    }
    // <<B_l | Q_pqr>> = S / (n^3 V^3)
    cudaError_t e = launch_modal_assemble(tfull, ufull, p->d_ells, (int)p->ells.size(), nf, (long long)nall, ntrip,
                                          1.0 / (n3 * V * V * V), S, st);
    if (e != cudaSuccess) return cuda_fail(e, "assemble (modal)");
    if ((ms = mark(p, st, 3)) != BSP_OK) return ms;
    p->launches_last = launches + 1;
    return BSP_OK;
}

bsp_status bsp_compute(bsp_plan* p, const void* delta_k, double nbar, void* ws, void* stream, double* B) {
    if (p && p->modal) return BSP_EINVAL;
    if (!p || !delta_k || !ws || !B || !aligned256(delta_k) || !aligned256(ws) || !aligned256(B) ||
        !(nbar >= 0) || !std::isfinite(nbar))
        return BSP_EINVAL;
    if (!p->have_counts) return BSP_ESTATE;
    return compute_impl(p, delta_k, nbar, ws, (cudaStream_t)stream, B);
}

bsp_status bsp_compute_host(bsp_plan* p, const void* delta_k_host, double nbar, void* ws, void* stream,
                            double* B_host) {
    if (!p || !delta_k_host || !ws || !B_host || !aligned256(ws) || !(nbar >= 0) || !std::isfinite(nbar))
        return BSP_EINVAL;
    if (!p->have_counts) return BSP_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    char* stage = (char*)ws + p->ws_bytes;
    const size_t dbytes = (size_t)p->n * p->n * (p->n / 2 + 1) * 8;
    double* Bdev = (double*)(stage + round256(dbytes));
    CK(cudaMemcpyAsync(stage, delta_k_host, dbytes, cudaMemcpyHostToDevice, st));
    bsp_status s = compute_impl(p, stage, nbar, ws, st, Bdev);
    if (s != BSP_OK) return s;
    CK(cudaMemcpyAsync(B_host, Bdev, sizeof(double) * p->ells.size() * p->bins.size(), cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
    return BSP_OK;
}

bsp_status bsp_device_status(bsp_plan* p, int* code) {
    if (!p || !code) return BSP_EINVAL;
    CK(cudaMemcpy(code, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return *code ? BSP_ETIMEOUT : BSP_OK;
}

bsp_status bsp_plan_stats(const bsp_plan* p, double* st) {
    if (!p || !st) return BSP_EINVAL;
    if (!p->have_counts) return BSP_ESTATE;
    double issued = 0, works = 0, nsplit = 1;
    if (p->tc) {
        for (const TcWork& w : p->tc_sched.works) issued += 128.0 * w.n * p->nprod;
        works = (double)p->tc_sched.works.size();
        nsplit = (double)p->tc_sched.units.size();
    } else {
        // 64 pairs times the 16-row blocks that hold rows (k_contract_cc32 skips the rest)
        for (const Work& w : p->comp_sched.works) issued += 64.0 * 16.0 * ((w.nrows + 15) / 16);
        works = (double)p->comp_sched.works.size();
        nsplit = p->comp_sched.nsplit;
    }
    st[0] = issued;
    st[1] = (double)p->ells.size() * p->bins.size();
    st[2] = works;
    st[3] = nsplit;
    return BSP_OK;
}

bsp_status bsp_plan_tune(bsp_plan* p, int target_ctas, int fft_batch) {
    if (!p || target_ctas < 0 || fft_batch < 0 || target_ctas > 4096) return BSP_EINVAL;
    if (fft_batch > 0) p->fb32 = std::min(fft_batch, p->fb_cap);
    if (target_ctas > 0 && target_ctas != p->target_ctas) {
        p->target_ctas = target_ctas;
        if (p->have_counts && !p->modal) return finish_counts(p);
    }
    return BSP_OK;
}

bsp_status bsp_plan_tune_tc(bsp_plan* p, int max_rows, int chunk_points) {
    if (!p || (max_rows && (max_rows < 32 || max_rows > 96 || max_rows % 8)) ||
        (chunk_points && (chunk_points < 64 || chunk_points % 64 || chunk_points > (1 << 20))))
        return BSP_EINVAL;
    if (!p->tc) return max_rows || chunk_points ? BSP_EUNSUPPORTED : BSP_OK;
    if (chunk_points) p->chunk_kb = chunk_points / 64;
    if (max_rows && max_rows / 8 != p->tc_max_boxes) {
        p->tc_max_boxes = max_rows / 8;
        if (p->have_counts && !p->modal) return finish_counts(p);
    }
    return BSP_OK;
}

bsp_status bsp_set_accumulation_chunk(bsp_plan* p, int points) {
    if (!p || points < 64 || points % 64 || points > (1 << 20)) return BSP_EINVAL;
    p->chunk_kb = points / 64;
    return BSP_OK;
}

bsp_status bsp_set_wait_limit(bsp_plan* p, long long cycles) {
    if (!p || cycles < 0 || cycles > (1ll << 40)) return BSP_EINVAL;
    p->wait_cycles = cycles;
    return BSP_OK;
}

bsp_status bsp_set_profiling(bsp_plan* p, int on) {
    if (!p) return BSP_EINVAL;
    p->profiling = on != 0;
    p->ev_used = 0;
    return BSP_OK;
}

bsp_status bsp_phase_times(bsp_plan* p, double* ms, int* ncalls, int* launches) {
    if (!p || !ms) return BSP_EINVAL;
    ms[0] = ms[1] = ms[2] = 0.0;
    const size_t calls = p->ev_used / 4;
    if (calls) CK(cudaEventSynchronize(p->ev_pool[4 * calls - 1]));
    for (size_t c = 0; c < calls; ++c)
        for (int k = 0; k < 3; ++k) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, p->ev_pool[4 * c + k], p->ev_pool[4 * c + k + 1]));
            ms[k] += t;
        }
    if (ncalls) *ncalls = (int)calls;
    if (launches) *launches = p->launches_last;
    p->ev_used = 0;
    return BSP_OK;
}

bsp_status bsp_power_compute(bsp_plan* p, const void* delta_k, double nbar, void* ws, void* stream, double* P,
                             double* Nk) {
    if (!p || !delta_k || !ws || !P || !aligned256(ws) || !(nbar >= 0.0)) return BSP_EINVAL;
    if (p->modal || p->nsh <= 0 || p->ells.size() > 3) return BSP_EINVAL;
    PowerEll pe{};
    pe.n = (int)p->ells.size();
    for (int i = 0; i < pe.n; ++i) pe.ell[i] = p->ells[i];
    // one FP64 slot per CTA at the start of the workspace (it fits: the
    // workspace holds at least one field per shell)
    const long long rows = (long long)p->geom.nK * p->geom.nK;
    int nblocks = (int)std::min<long long>(rows, 4LL * p->nsm);
    while (nblocks > 1 && power_partial_bytes(nblocks, p->nsh, pe.n) > p->ws_bytes) nblocks /= 2;
    if (power_partial_bytes(nblocks, p->nsh, pe.n) > p->ws_bytes) return BSP_ENOMEM;
    const double V = p->box * p->box * p->box;
    cudaError_t e = launch_power((const cx<float>*)delta_k, nullptr, 1.0, p->geom, p->d_shell_of, p->nsh, pe, V, nbar,
                                 nblocks, (double*)ws, P, Nk, (cudaStream_t)stream, 1, 0, 0, p->n2top);
    if (e != cudaSuccess) return cuda_fail(e, "power multipoles");
    return BSP_OK;
}

static bool density_geom(int n, FftGeom* g) {
    if (n < 8 || n % 2 != 0 || n > 2048) return false;
    *g = FftGeom{};
    g->n = n;
    g->K = n / 2;
    g->nK = n;
    g->pruned = 0;
    g->nKz = n / 2 + 1;
    g->n2max = 3 * (n / 2) * (n / 2);
    return radix_plan(n, g->rad, &g->nrad) && radix_plan(n / 2, g->rad_h, &g->nrad_h);
}

bsp_status bsp_density_workspace_size(int n, size_t* bytes) {
    FftGeom g;
    if (!bytes || !density_geom(n, &g)) return BSP_EINVAL;
    *bytes = density_layout(n).end;
    return BSP_OK;
}

bsp_status bsp_density_cic(int n, double box, long long n_particles, const float* pos, void* ws, size_t ws_bytes,
                           void* stream, void* delta_k, double* nbar) {
    FftGeom g;
    if (!density_geom(n, &g) || !(box > 0.0) || n_particles <= 0 || !pos || !ws || !delta_k || !aligned256(ws))
        return BSP_EINVAL;
    if (ws_bytes < density_layout(n).end) return BSP_ENOMEM;
    cudaError_t e = launch_density(g, pos, n_particles, box, ws, (cx<float>*)delta_k, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "density (CIC + forward FFT)");
    if (nbar) *nbar = (double)n_particles / (box * box * box);
    return BSP_OK;
}

// Skew-spectrum workspace: the real field x [n^3] FP32, then two unpruned
// half spectra (the inverse FFT's intermediates, reused for the transform of
// x^2 and for the per-CTA sums).
static size_t skew_bytes(int n, size_t* off_t1, size_t* off_t2) {
    const size_t x = round256((size_t)n * n * n * sizeof(float));
    const size_t h = round256((size_t)n * n * (n / 2 + 1) * sizeof(cx<float>));
    if (off_t1) *off_t1 = x;
    if (off_t2) *off_t2 = x + h;
    return x + 2 * h;
}

bsp_status bsp_skew_workspace_size(const bsp_plan* p, size_t* bytes) {
    if (!p || !bytes || p->modal) return BSP_EINVAL;
    *bytes = skew_bytes(p->n, nullptr, nullptr);
    return BSP_OK;
}

bsp_status bsp_skew_compute(bsp_plan* p, const void* delta_k, void* ws, size_t ws_bytes, void* stream, double* S,
                            double* Nk) {
    if (!p || !delta_k || !ws || !S || !aligned256(ws)) return BSP_EINVAL;
    if (p->modal || p->nsh <= 0 || p->ells.size() > 3 || !p->d_fd_raw) return BSP_EINVAL;
    FftGeom full;
    if (!density_geom(p->n, &full)) return BSP_EUNSUPPORTED;
    size_t o1, o2;
    if (ws_bytes < skew_bytes(p->n, &o1, &o2)) return BSP_ENOMEM;
    const cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    float* x = (float*)base;
    cx<float>* t1 = (cx<float>*)(base + o1);
    cx<float>* t2 = (cx<float>*)(base + o2);
    const size_t n3 = (size_t)p->n * p->n * p->n;
    // x = sum_{n != 0} delta(n) e^{ik.x} = V delta(x)
    cudaError_t e = launch_fft_fields<float>(full, (const cx<float>*)delta_k, p->d_shell_of, nullptr, p->d_fd_raw, 1,
                                             p->d_tw32, t1, t2, x, n3, nullptr, nullptr, 0, nullptr, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "skew (inverse FFT)");
    // transform of delta(x)^2 = x^2 / V^2, unnormalised, into t1
    const double V = p->box * p->box * p->box;
    e = launch_forward_square(full, x, (float)(1.0 / (V * V)), p->d_tw32, t1, st);
    if (e != cudaSuccess) return cuda_fail(e, "skew (forward FFT)");
    PowerEll pe{};
    pe.n = (int)p->ells.size();
    for (int i = 0; i < pe.n; ++i) pe.ell[i] = p->ells[i];
    const long long rows = (long long)p->geom.nK * p->geom.nK;
    int nblocks = (int)std::min<long long>(rows, 4LL * p->nsm);
    const size_t room = (size_t)(ws_bytes - o2);
    while (nblocks > 1 && power_partial_bytes(nblocks, p->nsh, pe.n) > room) nblocks /= 2;
    // Q = (V/n^3) x transform: the cross sum carries that factor
    e = launch_power((const cx<float>*)delta_k, t1, V / (double)n3, p->geom, p->d_shell_of, p->nsh, pe, V, 0.0,
                     nblocks, (double*)t2, S, Nk, st, 1, 0, 0, p->n2top);
    if (e != cudaSuccess) return cuda_fail(e, "skew (shell sums)");
    return BSP_OK;
}

// Integrated bispectrum (Sec. 3.4).  Workspace: the real field x [n^3] FP32,
// then one region used first by the inverse FFT's two half spectra and then
// by the m^3 sub-cube spectra, their twiddles and the per-CTA sums.
struct IbLayout {
    size_t t1, t2, sub, tw, part, end;
    int nbx;   // CTAs per cube of the shell sums
};

static bool ib_geom(const bsp_plan* p, int m, FftGeom* gs) {
    if (m < 1 || p->n % m != 0) return false;
    const int s = p->n / m;
    if (!density_geom(s, gs)) return false;
    // only |n_s| with m^2 |n_s|^2 below the top edge lie in a shell
    const double emax = p->edges.back();
    int K = 0;
    while ((double)(K + 1) * (K + 1) * m * m < emax * emax) ++K;
    if (K < s / 2) {
        gs->K = K;
        gs->nK = 2 * K + 1;
        gs->pruned = 1;
        gs->nKz = K + 1;
    }
    return true;
}

static IbLayout ib_layout(const bsp_plan* p, int m, const FftGeom& gs) {
    const int n = p->n, s = n / m, nc = m * m * m;
    IbLayout L{};
    const size_t x = round256((size_t)n * n * n * sizeof(float));
    const size_t h = round256((size_t)n * n * (n / 2 + 1) * sizeof(cx<float>));
    L.t1 = x;
    L.t2 = x + h;
    L.sub = x;
    L.tw = L.sub + round256((size_t)nc * s * s * (s / 2 + 1) * sizeof(cx<float>));
    L.part = L.tw + round256((size_t)s * sizeof(cx<float>));
    const long long rows = (long long)gs.nK * gs.nK;
    L.nbx = (int)std::max<long long>(1, std::min<long long>(rows / 8, (4LL * p->nsm + nc - 1) / nc));
    const size_t part = round256(power_partial_bytes(L.nbx * nc, p->nsh, (int)p->ells.size()));
    L.end = std::max(x + 2 * h, L.part + part);
    return L;
}

bsp_status bsp_ib_workspace_size(const bsp_plan* p, int m, size_t* bytes) {
    FftGeom gs;
    if (!p || !bytes || p->modal || !ib_geom(p, m, &gs) || m * m * m > 65535) return BSP_EINVAL;
    *bytes = ib_layout(p, m, gs).end;
    return BSP_OK;
}

bsp_status bsp_ib_compute(bsp_plan* p, const void* delta_k, int m, void* ws, size_t ws_bytes, void* stream,
                          double* iB, double* Nk) {
    if (!p || !delta_k || !ws || !iB || !aligned256(ws)) return BSP_EINVAL;
    if (p->modal || p->nsh <= 0 || p->ells.size() > 3 || !p->d_fd_raw || m < 1 || m * m * m > 65535)
        return BSP_EINVAL;
    FftGeom full, gs;
    if (!density_geom(p->n, &full)) return BSP_EUNSUPPORTED;
    if (!ib_geom(p, m, &gs)) return BSP_EUNSUPPORTED;
    const IbLayout L = ib_layout(p, m, gs);
    if (ws_bytes < L.end) return BSP_ENOMEM;
    if (p->ib_m != m) {   // shell table of the sub-cube grid, built once per m
        std::vector<int16_t> tab(gs.n2max + 1, -1);
        for (int q = 1; q <= gs.n2max; ++q) {
            const double n2 = (double)q * m * m;
            for (int a = 0; a < p->nsh; ++a)
                if (n2 >= p->edges[a] * p->edges[a] && n2 < p->edges[a + 1] * p->edges[a + 1]) {
                    tab[q] = (int16_t)a;
                    break;
                }
        }
        int top = 0;
        for (int q = 0; q <= gs.n2max; ++q)
            if (tab[q] >= 0) top = q;
        cudaFree(p->d_shell_sub);
        p->d_shell_sub = nullptr;
        p->ib_m = 0;
        bsp_status st = upload(&p->d_shell_sub, tab);
        if (st != BSP_OK) return st;
        p->ib_m = m;
        p->ib_n2top = top;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    float* x = (float*)base;
    const int n = p->n, s = n / m, nc = m * m * m;
    // x = sum_{n != 0} delta(n) e^{ik.x} = V delta(x)
    cudaError_t e = launch_fft_fields<float>(full, (const cx<float>*)delta_k, p->d_shell_of, nullptr, p->d_fd_raw, 1,
                                             p->d_tw32, (cx<float>*)(base + L.t1), (cx<float>*)(base + L.t2), x,
                                             (size_t)n * n * n, nullptr, nullptr, 0, nullptr, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "integrated bispectrum (inverse FFT)");
    // T_c = (1/(V s^3)) sum_{x in c} x e^{-ik.x}: T_c(0) is the cube mean of
    // delta, and the cube's own transform is delta_c(k) = V_s T_c(k)
    const double V = p->box * p->box * p->box, Vs = V / (double)nc;
    cx<float>* T = (cx<float>*)(base + L.sub);
    e = launch_forward_subcubes(gs, n, m, x, (float)(1.0 / (V * (double)s * s * s)), (cx<float>*)(base + L.tw), T, st);
    if (e != cudaSuccess) return cuda_fail(e, "integrated bispectrum (sub-cube FFTs)");
    PowerEll pe{};
    pe.n = (int)p->ells.size();
    for (int i = 0; i < pe.n; ++i) pe.ell[i] = p->ells[i];
    // iB^l_a = (1/m^3) sum_c T_c(0) (V_s^2 / (V_s N_a)) sum_{n in a} w_l |T_c|^2
    //        = V_s (sum_c T_c(0) sum w_l |T_c|^2) / (m^3 N_a)
    e = launch_power(T, nullptr, Vs, gs, p->d_shell_sub, p->nsh, pe, 1.0, 0.0, L.nbx, (double*)(base + L.part), iB,
                     Nk, st, nc, (size_t)s * s * (s / 2 + 1), 1, p->ib_n2top);
    if (e != cudaSuccess) return cuda_fail(e, "integrated bispectrum (shell sums)");
    return BSP_OK;
}

bsp_status bsp_last_raw(const bsp_plan* p, void* ws, void* stream, double* T) {
    if (!p || !ws || !T || !aligned256(ws)) return BSP_EINVAL;
    if (!p->have_counts) return BSP_ESTATE;
    const Layout L = layout_compute(p);
    CK(cudaMemcpyAsync(T, (char*)ws + L.tout, sizeof(double) * p->ells.size() * p->bins.size(),
                       cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return BSP_OK;
}

}  // extern "C"
