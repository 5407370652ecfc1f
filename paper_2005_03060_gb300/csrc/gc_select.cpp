// Reduced redundant-calibration selections (host side).
//
// Subset redundant calibration (paper Sec. 5): whole redundant groups in
// ascending order of baseline length until the pair count is the whole number
// of groups closest to p N log N (Eq. subredcal_frac_bls, Sec. 6.1), subject
// to the degeneracy criterion of Sec. 5.2.
// Low-cadence calibration (Sec. 4): every pair, p N log N pairs per
// integration cycle (Eq. lowcadcal_inttime), all pairs of a type in the same
// cycle, t_int = floor(T / N_cycle).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "gc_sel.h"

namespace {

struct TypeVec {
    int dx, dy;
};

// Canonical half-plane (dy > 0, or dy == 0 and dx > 0), ordered by squared
// length, ties by angle in [0, pi) -- compared exactly with a cross product.
std::vector<TypeVec> ordered_types(int L) {
    std::vector<TypeVec> t;
    for (int dy = 0; dy < L; ++dy)
        for (int dx = -(L - 1); dx < L; ++dx)
            if (dy > 0 || dx > 0) t.push_back({dx, dy});
    std::stable_sort(t.begin(), t.end(), [](const TypeVec &a, const TypeVec &b) {
        const long la = (long)a.dx * a.dx + (long)a.dy * a.dy;
        const long lb = (long)b.dx * b.dx + (long)b.dy * b.dy;
        if (la != lb) return la < lb;
        // both angles lie in [0, pi): a before b iff cross(a, b) > 0
        return (long)a.dx * b.dy - (long)a.dy * b.dx > 0;
    });
    return t;
}

int group_size(int L, const TypeVec &d) { return (L - std::abs(d.dx)) * (L - std::abs(d.dy)); }

double pair_budget(int N, double p, double log_base) {
    const double lg = log_base > 0.0 ? std::log((double)N) / std::log(log_base) : std::log((double)N);
    return p * N * lg;
}

// Null-space dimension of the linearised system for a prefix of the ordered
// types on an L x L grid with L >= 3: the phase part keeps its three
// directions (offset and two slopes) once (1,0) and (0,1) are present; the
// amplitude part keeps only the overall scale once a type with dx + dy even
// couples antennas of equal checkerboard parity (without one, the
// checkerboard amplitude pattern is a fifth direction).  A set lacking an
// axis type is reported as 6 (not a valid calibration set).
int null_dim_of(int L, const std::vector<TypeVec> &types) {
    if (L < 3) return 6;
    bool x = false, y = false, even = false;
    for (const auto &d : types) {
        if (d.dx == 1 && d.dy == 0) x = true;
        if (d.dx == 0 && d.dy == 1) y = true;
        if (((d.dx + d.dy) & 1) == 0) even = true;
    }
    if (!x || !y) return 6;
    return even ? 4 : 5;
}

void fill_pairs(gc_sel *s) {
    const int L = s->L;
    s->type_ptr.assign(1, 0);
    s->pair_i.clear();
    s->pair_j.clear();
    s->pair_type.clear();
    for (int k = 0; k < s->n_ubl; ++k) {
        const int dx = s->types[2 * k], dy = s->types[2 * k + 1];
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                const int xi = x + dx, yi = y + dy;
                if (xi < 0 || xi >= L || yi < 0 || yi >= L) continue;
                if (s->masked && !(s->mask[yi * L + xi] && s->mask[y * L + x])) continue;
                s->pair_i.push_back(yi * L + xi);
                s->pair_j.push_back(y * L + x);
                s->pair_type.push_back(k);
            }
        s->type_ptr.push_back((int32_t)s->pair_i.size());
    }
    s->P = (int)s->pair_i.size();
    const size_t N = (size_t)L * L;
    s->nbr.clear();
    if (2 * (size_t)s->n_ubl * N <= (16u << 20)) {
        s->nbr.assign(2 * (size_t)s->n_ubl * N, -1);
        for (int q = 0; q < s->P; ++q) {
            const int k = s->pair_type[q];
            s->nbr[(size_t)k * N + s->pair_i[q]] = q;
            s->nbr[(size_t)(s->n_ubl + k) * N + s->pair_j[q]] = q;
        }
    }
}

// X-engine work groups: types that share a window, at most GC_XENG_NTY each.
void fill_groups(gc_sel *s) {
    s->grp_types.clear();
    s->grp_off.assign(1, 0);
    s->grp_t0.clear();
    s->grp_t1.clear();
    s->grp_first.clear();
    s->grp_win.clear();
    s->grp_dymax.clear();
    std::vector<int> order(s->n_ubl);
    for (int k = 0; k < s->n_ubl; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s->win_t0[a] < s->win_t0[b]; });
    int k = 0;
    s->n_windows = 0;
    while (k < s->n_ubl) {
        const int t0 = s->win_t0[order[k]], t1 = s->win_t1[order[k]];
        bool first = true;
        while (k < s->n_ubl && s->win_t0[order[k]] == t0) {
            int n = 0, dymax = 0;
            while (k < s->n_ubl && s->win_t0[order[k]] == t0 && n < GC_XENG_NTY) {
                s->grp_types.push_back(order[k]);
                dymax = std::max(dymax, s->types[2 * order[k] + 1]);
                ++k;
                ++n;
            }
            s->grp_dymax.push_back(dymax);
            s->grp_off.push_back((int32_t)s->grp_types.size());
            s->grp_t0.push_back(t0);
            s->grp_t1.push_back(t1);
            s->grp_first.push_back(first ? 1 : 0);
            s->grp_win.push_back(s->n_windows);
            first = false;
        }
        ++s->n_windows;
    }
    s->n_groups = (int)s->grp_t0.size();
}

// Types with at least one pair between occupied points of `mask`, with
// their pair counts, ordered by physical length on the lattice (square:
// dx^2 + dy^2; triangular, basis (1,0), (1/2, sqrt3/2): dx^2 + dx dy + dy^2),
// ties by angle in [0, pi) (the lattice map preserves orientation, so the
// lattice cross product orders the angles).
std::vector<std::pair<TypeVec, long>> masked_types(int L, const std::vector<int32_t> &mask, int lattice) {
    std::vector<std::pair<TypeVec, long>> t;
    for (int dy = 0; dy < L; ++dy)
        for (int dx = -(L - 1); dx < L; ++dx) {
            if (!(dy > 0 || dx > 0)) continue;
            long n = 0;
            for (int y = std::max(0, -dy); y < std::min(L, L - dy); ++y)
                for (int x = std::max(0, -dx); x < std::min(L, L - dx); ++x)
                    n += mask[y * L + x] && mask[(y + dy) * L + x + dx];
            if (n > 0) t.push_back({{dx, dy}, n});
        }
    auto len2 = [lattice](const TypeVec &d) {
        return lattice ? (long)d.dx * d.dx + (long)d.dx * d.dy + (long)d.dy * d.dy
                       : (long)d.dx * d.dx + (long)d.dy * d.dy;
    };
    std::stable_sort(t.begin(), t.end(), [&](const std::pair<TypeVec, long> &a, const std::pair<TypeVec, long> &b) {
        const long la = len2(a.first), lb = len2(b.first);
        if (la != lb) return la < lb;
        return (long)a.first.dx * b.first.dy - (long)a.first.dy * b.first.dx > 0;
    });
    return t;
}

// Start-point tree of a masked selection: breadth-first over the pairs of the
// (1,0) and (0,1) types from the first occupied point.  False when these
// types do not connect every occupied point.
bool fill_tree(gc_sel *s) {
    const int L = s->L, N = L * L;
    int ax = -1, ay = -1;
    for (int k = 0; k < s->n_ubl; ++k) {
        if (s->types[2 * k] == 1 && s->types[2 * k + 1] == 0) ax = k;
        if (s->types[2 * k] == 0 && s->types[2 * k + 1] == 1) ay = k;
    }
    if (ax < 0 || ay < 0 || s->nbr.empty()) return false;
    s->tree_ant.clear();
    s->tree_pair.clear();
    s->tree_sign.clear();
    std::vector<char> seen(N, 0);
    int root = 0;
    while (root < N && !s->mask[root]) ++root;
    if (root == N) return false;
    seen[root] = 1;
    s->tree_ant.push_back(root);
    s->tree_pair.push_back(-1);
    s->tree_sign.push_back(0);
    for (size_t h = 0; h < s->tree_ant.size(); ++h) {
        const int a = s->tree_ant[h];
        for (int k : {ax, ay}) {
            for (int role = 0; role < 2; ++role) {
                // role 0: a is the first member, the partner the second; role 1: the reverse
                const int q = s->nbr[(size_t)(role * s->n_ubl + k) * N + a];
                if (q < 0) continue;
                const int b = role == 0 ? s->pair_j[q] : s->pair_i[q];
                if (seen[b]) continue;
                seen[b] = 1;
                s->tree_ant.push_back(b);
                s->tree_pair.push_back(q);
                s->tree_sign.push_back(role == 0 ? -1 : 1);   // b second member: -1; first: +1
            }
        }
    }
    return (int)s->tree_ant.size() == s->n_occ;
}

// Largest selection the builders hold: 2^28 pairs (3.2 GB of host pair
// arrays, as much again on the device).  Low-cadence selections take every
// pair, N (N - 1) / 2, so they stop at about 23 000 antennas.
constexpr long kMaxPairs = 1L << 28;

// No C++ exception leaves the C ABI: allocation failure reads GC_ENOMEM.
template <class F>
gc_status no_throw(F &&f) {
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return GC_ENOMEM;
    } catch (...) {
        return GC_EINVAL;
    }
}

}  // namespace

void gc_sel_release_device(gc_sel *s) {
    if (!s || !s->d_base) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    cudaFree(s->d_base);
    cudaSetDevice(prev);
    s->d_base = nullptr;
}

gc_status gc_sel_upload(gc_ctx *ctx, gc_sel *s) {
    if (s->d_base && s->device == ctx->device) return GC_OK;
    gc_sel_release_device(s);
    // one allocation: types, type_ptr, pair_i, pair_j, pair_type, win_t0, win_t1, grp_* arrays
    const std::vector<int32_t> *parts[] = {&s->types,    &s->type_ptr,  &s->pair_i,    &s->pair_j,
                                           &s->pair_type, &s->win_t0,   &s->win_t1,    &s->grp_types,
                                           &s->grp_off,  &s->grp_t0,    &s->grp_t1,    &s->grp_first,
                                           &s->grp_win,  &s->nbr,       &s->grp_dymax, &s->mask,
                                           &s->tree_ant, &s->tree_pair, &s->tree_sign};
    constexpr int kParts = 19;
    size_t total = 0;
    size_t offs[kParts];
    for (int i = 0; i < kParts; ++i) {
        offs[i] = total;
        total += ((parts[i]->size() * sizeof(int32_t) + 255) / 256) * 256;
    }
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, std::max<size_t>(total, 256));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return gc_cuda_fail(ctx, e, "cudaMalloc(selection)");
    }
    for (int i = 0; i < kParts; ++i) {
        if (parts[i]->empty()) continue;
        e = cudaMemcpy(static_cast<char *>(base) + offs[i], parts[i]->data(), parts[i]->size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(base);
            return gc_cuda_fail(ctx, e, "upload selection");
        }
    }
    int32_t **dst[] = {&s->d_types,    &s->d_type_ptr,  &s->d_pair_i,    &s->d_pair_j,
                       &s->d_pair_type, &s->d_win_t0,   &s->d_win_t1,    &s->d_grp_types,
                       &s->d_grp_off,  &s->d_grp_t0,    &s->d_grp_t1,    &s->d_grp_first,
                       &s->d_grp_win,  &s->d_nbr,       &s->d_grp_dymax, &s->d_mask,
                       &s->d_tree_ant, &s->d_tree_pair, &s->d_tree_sign};
    for (int i = 0; i < kParts; ++i)
        *dst[i] = parts[i]->empty() ? nullptr : reinterpret_cast<int32_t *>(static_cast<char *>(base) + offs[i]);
    s->d_base = base;
    s->device = ctx->device;
    return GC_OK;
}

extern "C" {

static gc_status gc_selection_subset_impl(int L, int T, double p, double log_base, gc_sel **out) {
    if (!out) return GC_EINVAL;
    *out = nullptr;
    if (L == 2) return GC_EDEGEN;   // 6 visibilities for 8 unknowns: never four degeneracies
    if (L < 3 || L > 256 || T < 1 || !(p > 0.0) || log_base < 0.0 || log_base == 1.0) return GC_EINVAL;
    const std::vector<TypeVec> ord = ordered_types(L);
    const double target = pair_budget(L * L, p, log_base);
    long cum = 0;
    int best_k = 1;
    double best_err = -1.0;
    for (size_t k = 0; k < ord.size(); ++k) {
        cum += group_size(L, ord[k]);
        const double err = std::fabs((double)cum - target);
        if (best_err < 0.0 || err < best_err) {
            best_err = err;
            best_k = (int)k + 1;
        }
    }
    // extend until the degeneracy criterion holds (Sec. 5.2)
    int k = best_k;
    while (k < (int)ord.size() && null_dim_of(L, std::vector<TypeVec>(ord.begin(), ord.begin() + k)) != 4) ++k;
    std::vector<TypeVec> chosen(ord.begin(), ord.begin() + k);
    const int nd = null_dim_of(L, chosen);
    if (nd != 4) return GC_EDEGEN;
    std::unique_ptr<gc_sel> s(new (std::nothrow) gc_sel());
    if (!s) return GC_ENOMEM;
    s->scheme = 0;
    s->L = L;
    s->T = T;
    s->n_occ = L * L;
    s->n_ubl = k;
    s->n_cycle = 1;
    s->t_int = T;
    s->null_dim = nd;
    s->target = target;
    for (const auto &d : chosen) {
        s->types.push_back(d.dx);
        s->types.push_back(d.dy);
        s->win_t0.push_back(0);
        s->win_t1.push_back(T);
    }
    fill_pairs(s.get());
    fill_groups(s.get());
    *out = s.release();
    return GC_OK;
}

static gc_status gc_selection_lowcad_impl(int L, int T, double p, double log_base, gc_sel **out) {
    if (!out) return GC_EINVAL;
    *out = nullptr;
    if (L < 3 || L > 256 || T < 1 || !(p > 0.0) || log_base < 0.0 || log_base == 1.0) return GC_EINVAL;
    const std::vector<TypeVec> ord = ordered_types(L);
    const double target = pair_budget(L * L, p, log_base);
    const long cap = (long)std::floor(target);
    std::vector<long> room;        // free capacity per cycle
    std::vector<int> cycle(ord.size());
    for (size_t k = 0; k < ord.size(); ++k) {
        const long n = group_size(L, ord[k]);
        if (n > cap) return GC_EINVAL;   // a redundant group must fit one cycle
        size_t c = 0;
        while (c < room.size() && room[c] < n) ++c;
        if (c == room.size()) room.push_back(cap);
        room[c] -= n;
        cycle[k] = (int)c;
    }
    const int n_cycle = (int)room.size();
    const int t_int = T / n_cycle;
    if (t_int < 1) return GC_EINVAL;     // integration too short for the cycle count
    if ((long)L * L * ((long)L * L - 1) / 2 > kMaxPairs) return GC_EUNSUPPORTED;
    std::unique_ptr<gc_sel> s(new (std::nothrow) gc_sel());
    if (!s) return GC_ENOMEM;
    s->scheme = 1;
    s->L = L;
    s->T = T;
    s->n_occ = L * L;
    s->n_ubl = (int)ord.size();
    s->n_cycle = n_cycle;
    s->t_int = t_int;
    s->null_dim = null_dim_of(L, ord);
    s->target = target;
    for (size_t k = 0; k < ord.size(); ++k) {
        s->types.push_back(ord[k].dx);
        s->types.push_back(ord[k].dy);
        s->win_t0.push_back(cycle[k] * t_int);
        s->win_t1.push_back((cycle[k] + 1) * t_int);
    }
    fill_pairs(s.get());
    fill_groups(s.get());
    *out = s.release();
    return GC_OK;
}

static gc_status gc_selection_subset_masked_impl(int L, int T, double p, double log_base, const uint8_t *mask, int lattice,
                                     gc_sel **out) {
    if (!out) return GC_EINVAL;
    *out = nullptr;
    if (!mask || L < 3 || L > 256 || T < 1 || !(p > 0.0) || log_base < 0.0 || log_base == 1.0 ||
        (lattice != GC_LATTICE_SQUARE && lattice != GC_LATTICE_TRIANGULAR))
        return GC_EINVAL;
    std::vector<int32_t> m((size_t)L * L);
    int n_occ = 0;
    for (int i = 0; i < L * L; ++i) n_occ += (m[i] = mask[i] ? 1 : 0);
    if (n_occ < 3) return GC_EINVAL;
    const auto ord = masked_types(L, m, lattice);
    const double target = pair_budget(n_occ, p, log_base);
    long cum = 0;
    int best_k = 1;
    double best_err = -1.0;
    for (size_t k = 0; k < ord.size(); ++k) {
        cum += ord[k].second;
        const double err = std::fabs((double)cum - target);
        if (best_err < 0.0 || err < best_err) {
            best_err = err;
            best_k = (int)k + 1;
        }
    }
    // degeneracy criterion (Sec. 5.2) by rule: both axis types, and a type
    // that breaks the checkerboard amplitude pattern -- dx + dy even on the
    // square lattice, (-1, 1) on the triangular one (the third unit direction)
    auto criterion = [&](int k) {
        bool x = false, y = false, odd_cycle = false;
        for (int q = 0; q < k; ++q) {
            const TypeVec &d = ord[q].first;
            if (d.dx == 1 && d.dy == 0) x = true;
            if (d.dx == 0 && d.dy == 1) y = true;
            if (lattice == GC_LATTICE_SQUARE ? ((d.dx + d.dy) & 1) == 0 : (d.dx == -1 && d.dy == 1)) odd_cycle = true;
        }
        return x && y && odd_cycle;
    };
    int k = best_k;
    while (k < (int)ord.size() && !criterion(k)) ++k;
    if (!criterion(k)) return GC_EDEGEN;
    std::unique_ptr<gc_sel> s(new (std::nothrow) gc_sel());
    if (!s) return GC_ENOMEM;
    s->scheme = 0;
    s->L = L;
    s->T = T;
    s->n_ubl = k;
    s->n_cycle = 1;
    s->t_int = T;
    s->null_dim = 4;
    s->target = target;
    s->lattice = lattice;
    s->masked = 1;
    s->n_occ = n_occ;
    s->mask = m;
    for (int q = 0; q < k; ++q) {
        s->types.push_back(ord[q].first.dx);
        s->types.push_back(ord[q].first.dy);
        s->win_t0.push_back(0);
        s->win_t1.push_back(T);
    }
    fill_pairs(s.get());
    fill_groups(s.get());
    if (!fill_tree(s.get())) {   // the axis types must connect the array
        return GC_EDEGEN;
    }
    *out = s.release();
    return GC_OK;
}

static gc_status gc_selection_lowcad_masked_impl(int L, int T, double p, double log_base, const uint8_t *mask, int lattice,
                                     gc_sel **out) {
    if (!out) return GC_EINVAL;
    *out = nullptr;
    if (!mask || L < 3 || L > 256 || T < 1 || !(p > 0.0) || log_base < 0.0 || log_base == 1.0 ||
        (lattice != GC_LATTICE_SQUARE && lattice != GC_LATTICE_TRIANGULAR))
        return GC_EINVAL;
    std::vector<int32_t> m((size_t)L * L);
    int n_occ = 0;
    for (int i = 0; i < L * L; ++i) n_occ += (m[i] = mask[i] ? 1 : 0);
    if (n_occ < 3) return GC_EINVAL;
    const auto ord = masked_types(L, m, lattice);
    const double target = pair_budget(n_occ, p, log_base);
    const long cap = (long)std::floor(target);
    std::vector<long> room;
    std::vector<int> cycle(ord.size());
    for (size_t k = 0; k < ord.size(); ++k) {   // first-fit of whole types, shortest first
        const long n = ord[k].second;
        if (n > cap) return GC_EINVAL;
        size_t c = 0;
        while (c < room.size() && room[c] < n) ++c;
        if (c == room.size()) room.push_back(cap);
        room[c] -= n;
        cycle[k] = (int)c;
    }
    const int n_cycle = (int)room.size();
    const int t_int = T / n_cycle;
    if (t_int < 1) return GC_EINVAL;
    if ((long)n_occ * (n_occ - 1) / 2 > kMaxPairs) return GC_EUNSUPPORTED;
    std::unique_ptr<gc_sel> s(new (std::nothrow) gc_sel());
    if (!s) return GC_ENOMEM;
    s->scheme = 1;
    s->L = L;
    s->T = T;
    s->n_ubl = (int)ord.size();
    s->n_cycle = n_cycle;
    s->t_int = t_int;
    s->null_dim = 4;   // every type is in: the criterion holds when the array is connected (checked below)
    s->target = target;
    s->lattice = lattice;
    s->masked = 1;
    s->n_occ = n_occ;
    s->mask = m;
    bool x = false, y = false;
    for (size_t k = 0; k < ord.size(); ++k) {
        s->types.push_back(ord[k].first.dx);
        s->types.push_back(ord[k].first.dy);
        s->win_t0.push_back(cycle[k] * t_int);
        s->win_t1.push_back((cycle[k] + 1) * t_int);
        x = x || (ord[k].first.dx == 1 && ord[k].first.dy == 0);
        y = y || (ord[k].first.dx == 0 && ord[k].first.dy == 1);
    }
    fill_pairs(s.get());
    fill_groups(s.get());
    if (!x || !y || !fill_tree(s.get())) {
        return GC_EDEGEN;
    }
    *out = s.release();
    return GC_OK;
}

gc_status gc_selection_subset(int L, int T, double p, double log_base, gc_sel **out) {
    if (out) *out = nullptr;
    return no_throw([&] { return gc_selection_subset_impl(L, T, p, log_base, out); });
}

gc_status gc_selection_lowcad(int L, int T, double p, double log_base, gc_sel **out) {
    if (out) *out = nullptr;
    return no_throw([&] { return gc_selection_lowcad_impl(L, T, p, log_base, out); });
}

gc_status gc_selection_subset_masked(int L, int T, double p, double log_base, const uint8_t *mask, int lattice,
                                     gc_sel **out) {
    if (out) *out = nullptr;
    return no_throw([&] { return gc_selection_subset_masked_impl(L, T, p, log_base, mask, lattice, out); });
}

gc_status gc_selection_lowcad_masked(int L, int T, double p, double log_base, const uint8_t *mask, int lattice,
                                     gc_sel **out) {
    if (out) *out = nullptr;
    return no_throw([&] { return gc_selection_lowcad_masked_impl(L, T, p, log_base, mask, lattice, out); });
}

void gc_sel_free(gc_sel *sel) {
    if (!sel) return;
    gc_sel_release_device(sel);
    delete sel;
}

gc_status gc_sel_info(const gc_sel *s, int32_t *info) {
    if (!s || !info) return GC_EINVAL;
    info[0] = s->L;
    info[1] = s->T;
    info[2] = s->P;
    info[3] = s->n_ubl;
    info[4] = s->n_cycle;
    info[5] = s->t_int;
    info[6] = s->null_dim;
    info[7] = s->scheme;
    info[8] = s->masked;
    info[9] = s->lattice;
    info[10] = s->n_occ;
    return GC_OK;
}

gc_status gc_sel_arrays(const gc_sel *s, const int32_t **types, const int32_t **type_ptr, const int32_t **pair_i,
                        const int32_t **pair_j, const int32_t **win_t0, const int32_t **win_t1) {
    if (!s) return GC_EINVAL;
    if (types) *types = s->types.data();
    if (type_ptr) *type_ptr = s->type_ptr.data();
    if (pair_i) *pair_i = s->pair_i.data();
    if (pair_j) *pair_j = s->pair_j.data();
    if (win_t0) *win_t0 = s->win_t0.data();
    if (win_t1) *win_t1 = s->win_t1.data();
    return GC_OK;
}

gc_status gc_sel_edge(const gc_sel *s, uint8_t *edge) {
    if (!s || !edge) return GC_EINVAL;
    // nearest-neighbour steps: 4 on the square lattice; the triangular
    // lattice is stored sheared, its other two neighbours at (1, -1), (-1, 1)
    static const int kStep[6][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1}};
    const int n_step = s->lattice == 1 ? 6 : 4;
    const int L = s->L;
    auto occ = [&](int x, int y) {
        return x >= 0 && x < L && y >= 0 && y < L && (!s->masked || s->mask[(size_t)y * L + x] != 0);
    };
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            uint8_t e = 0;
            if (occ(x, y))
                for (int k = 0; k < n_step; ++k)
                    if (!occ(x + kStep[k][0], y + kStep[k][1])) e = 1;
            edge[(size_t)y * L + x] = e;
        }
    return GC_OK;
}

}  // extern "C"
