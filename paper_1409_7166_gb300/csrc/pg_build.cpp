// Host-side grid builder: validation (Section III-B), sub-circuit split
// (Fig. 1), colouring for the parallel Gauss-Seidel order, and SELL packing.
//
// Nothing here depends on the time step h; per-h coefficients are assembled
// in pg_api.cu from the merged neighbour lists built here.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>

#include "pg_internal.h"

namespace pg {

namespace {

struct Dsu {
    std::vector<int32_t> p;
    explicit Dsu(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
    int find(int x) {
        while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
        return x;
    }
    void unite(int a, int b) {
        a = find(a); b = find(b);
        if (a != b) p[std::max(a, b)] = std::min(a, b);
    }
};

inline bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

void pwl_aux(const std::vector<int64_t>& ptr, const std::vector<double>& t, const std::vector<double>& v,
             std::vector<double>* slope, std::vector<unsigned long long>* key) {
    slope->assign(t.size(), 0.0);
    key->assign(t.size(), 0ull);
    for (size_t e = 0; e + 1 < ptr.size(); ++e)
        for (int64_t k = ptr[e]; k < ptr[e + 1]; ++k) {
            if (k + 1 < ptr[e + 1] && t[k + 1] > t[k]) (*slope)[k] = (v[k + 1] - v[k]) / (t[k + 1] - t[k]);
            uint64_t b;
            std::memcpy(&b, &t[k], sizeof b);
            (*key)[k] = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
        }
}

pg_status build_packed(const pg_netlist* nl, Packed* P, std::string* why, int32_t lattice_policy, int32_t colouring) {
    auto fail = [&](pg_status s, const std::string& m) { if (why) *why = m; return s; };
    if (!nl || !P) return fail(PG_ERR_INVALID_ARG, "null netlist");
    const int32_t n = nl->n_nodes, p = nl->n_sources;
    if (n < 1 || p < 0) return fail(PG_ERR_INVALID_ARG, "n_nodes < 1 or n_sources < 0");
    if (nl->n_r < 0 || nl->n_c < 0 || nl->n_l < 0 || nl->n_i < 0)
        return fail(PG_ERR_INVALID_ARG, "negative element count");
    if ((p && !nl->vdd) || (nl->n_r && (!nl->r_a || !nl->r_b || !nl->r_g)) ||
        (nl->n_c && (!nl->c_a || !nl->c_b || !nl->c_val)) ||
        (nl->n_l && (!nl->l_a || !nl->l_b || !nl->l_val)) ||
        (nl->n_i && (!nl->i_a || !nl->i_b || !nl->i_ptr || !nl->i_t || !nl->i_v)))
        return fail(PG_ERR_INVALID_ARG, "null element array");
    for (int k = 0; k < p; ++k)
        if (!std::isfinite(nl->vdd[k])) return fail(PG_ERR_INVALID_ARG, "non-finite vdd");
    auto term_ok = [&](int32_t t) { return (t >= 0 && t < n) || t == PG_GROUND || (t <= -2 && -2 - t < p); };

    P->n = n; P->p = p;
    P->vdd.assign(nl->vdd, nl->vdd + p);
    std::vector<int32_t> deg(n, 0);       // non-current-source branches per node (assumption 2)

    // --- merged neighbour lists: count, fill, sort, merge
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t e = 0; e < nl->n_r; ++e) {
        int32_t a = nl->r_a[e], b = nl->r_b[e];
        if (!term_ok(a) || !term_ok(b)) return fail(PG_ERR_INVALID_ARG, "resistor terminal out of range");
        if (a == b) return fail(PG_ERR_INVALID_ARG, "resistor with both terminals equal");
        if (!finite_pos(nl->r_g[e])) return fail(PG_ERR_INVALID_ARG, "resistor conductance must be > 0");
        if (a >= 0 && b >= 0) { cnt[a + 1]++; cnt[b + 1]++; }
    }
    for (int64_t e = 0; e < nl->n_l; ++e) {
        int32_t a = nl->l_a[e], b = nl->l_b[e];
        if (!term_ok(a) || !term_ok(b)) return fail(PG_ERR_INVALID_ARG, "inductor terminal out of range");
        if (a == b) return fail(PG_ERR_INVALID_ARG, "inductor with both terminals equal");
        if (!finite_pos(nl->l_val[e])) return fail(PG_ERR_INVALID_ARG, "inductance must be > 0");
        if (a >= 0 && b >= 0) { cnt[a + 1]++; cnt[b + 1]++; }
    }
    for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> tn(cnt[n]);
    std::vector<double> tg(cnt[n]), tl(cnt[n]);
    std::vector<int64_t> fillp(cnt.begin(), cnt.end() - 1);
    P->g_gnd.assign(n, 0.0); P->il_gnd.assign(n, 0.0); P->cap.assign(n, 0.0);
    P->inj_g.assign(n, 0.0); P->inj_il.assign(n, 0.0);
    auto tv = [&](int32_t t) { return t == PG_GROUND ? 0.0 : nl->vdd[-2 - t]; };
    Dsu dsu(n);
    std::vector<uint8_t> r_anchor(n, 0), any_anchor(n, 0);
    for (int64_t e = 0; e < nl->n_r; ++e) {
        int32_t a = nl->r_a[e], b = nl->r_b[e];
        double g = nl->r_g[e];
        if (a >= 0 && b >= 0) {
            int64_t k = fillp[a]++; tn[k] = b; tg[k] = g; tl[k] = 0.0;
            k = fillp[b]++; tn[k] = a; tg[k] = g; tl[k] = 0.0;
            dsu.unite(a, b); deg[a]++; deg[b]++;
        } else if (a >= 0 || b >= 0) {
            int32_t i = a >= 0 ? a : b, o = a >= 0 ? b : a;
            P->g_gnd[i] += g; P->inj_g[i] += g * tv(o);
            r_anchor[i] = any_anchor[i] = 1; deg[i]++;
        }
    }
    for (int64_t e = 0; e < nl->n_l; ++e) {
        int32_t a = nl->l_a[e], b = nl->l_b[e];
        double il = 1.0 / nl->l_val[e];
        if (a >= 0 && b >= 0) {
            int64_t k = fillp[a]++; tn[k] = b; tg[k] = 0.0; tl[k] = il;
            k = fillp[b]++; tn[k] = a; tg[k] = 0.0; tl[k] = il;
            dsu.unite(a, b); deg[a]++; deg[b]++;
        } else if (a >= 0 || b >= 0) {
            int32_t i = a >= 0 ? a : b, o = a >= 0 ? b : a;
            P->il_gnd[i] += il; P->inj_il[i] += il * tv(o);
            any_anchor[i] = 1; deg[i]++;
        }
    }
    for (int64_t e = 0; e < nl->n_c; ++e) {
        int32_t a = nl->c_a[e], b = nl->c_b[e];
        if (!term_ok(a) || !term_ok(b)) return fail(PG_ERR_INVALID_ARG, "capacitor terminal out of range");
        if (!finite_pos(nl->c_val[e])) return fail(PG_ERR_INVALID_ARG, "capacitance must be > 0");
        if (a >= 0 && b >= 0)
            return fail(PG_ERR_UNSUPPORTED, "node-to-node capacitor: only grounded C_i fit the per-node form (Eq. 12)");
        if (a >= 0 || b >= 0) { int32_t i = a >= 0 ? a : b; P->cap[i] += nl->c_val[e]; deg[i]++; }
    }
    // current sources
    if (nl->n_i) {
        if (nl->i_ptr[0] != 0) return fail(PG_ERR_INVALID_ARG, "i_ptr[0] must be 0");
        for (int64_t e = 0; e < nl->n_i; ++e) {
            if (!term_ok(nl->i_a[e]) || !term_ok(nl->i_b[e]))
                return fail(PG_ERR_INVALID_ARG, "current source terminal out of range");
            int64_t s0 = nl->i_ptr[e], s1 = nl->i_ptr[e + 1];
            if (s1 <= s0) return fail(PG_ERR_INVALID_ARG, "current source without breakpoints");
            for (int64_t k = s0; k < s1; ++k) {
                if (!std::isfinite(nl->i_t[k]) || !std::isfinite(nl->i_v[k]))
                    return fail(PG_ERR_INVALID_ARG, "non-finite PWL breakpoint");
                if (k > s0 && nl->i_t[k] < nl->i_t[k - 1])
                    return fail(PG_ERR_INVALID_ARG, "PWL breakpoint times must be non-decreasing");
            }
        }
    }
    for (int i = 0; i < n; ++i)
        if (deg[i] == 0)
            return fail(PG_ERR_FLOATING_NODE, "node " + std::to_string(i) +
                        " has no resistor, capacitor or inductor (topological assumption 2)");

    // components: each must reach a source or ground through R or L
    P->comp_of.assign(n, 0);
    std::vector<int32_t> root_id(n, -1);
    int32_t ncomp = 0;
    for (int i = 0; i < n; ++i) {
        int r = dsu.find(i);
        if (root_id[r] < 0) root_id[r] = ncomp++;
        P->comp_of[i] = root_id[r];
    }
    P->n_comp = ncomp;
    std::vector<uint8_t> comp_any(ncomp, 0);
    P->comp_has_r_anchor.assign(ncomp, 0);
    for (int i = 0; i < n; ++i) {
        comp_any[P->comp_of[i]] |= any_anchor[i];
        P->comp_has_r_anchor[P->comp_of[i]] |= r_anchor[i];
    }
    for (int c = 0; c < ncomp; ++c)
        if (!comp_any[c]) {
            int first = 0;
            while (P->comp_of[first] != c) ++first;
            return fail(PG_ERR_FLOATING_NODE, "sub-circuit containing node " + std::to_string(first) +
                        " has no resistor or inductor to a source or ground (floating)");
        }

    // sort + merge each node's neighbours (parallel R||L on one pair becomes one weight)
    P->adj_ptr.assign(n + 1, 0);
    P->adj_nbr.clear(); P->adj_g.clear(); P->adj_il.clear();
    P->adj_nbr.reserve(cnt[n]); P->adj_g.reserve(cnt[n]); P->adj_il.reserve(cnt[n]);
    std::vector<int64_t> ord;
    for (int i = 0; i < n; ++i) {
        int64_t s0 = cnt[i], s1 = cnt[i + 1];
        ord.resize(s1 - s0);
        std::iota(ord.begin(), ord.end(), s0);
        std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return tn[x] < tn[y]; });
        for (size_t k = 0; k < ord.size(); ++k) {
            int64_t e = ord[k];
            if (k > 0 && tn[e] == P->adj_nbr.back()) {
                P->adj_g.back() += tg[e]; P->adj_il.back() += tl[e];
            } else {
                P->adj_nbr.push_back(tn[e]); P->adj_g.push_back(tg[e]); P->adj_il.push_back(tl[e]);
            }
        }
        P->adj_ptr[i + 1] = (int64_t)P->adj_nbr.size();
    }
    { std::vector<int32_t>().swap(tn); std::vector<double>().swap(tg); std::vector<double>().swap(tl); }

    // --- lattice form: lattices cover every node and every merged neighbour pair is a
    //     lattice neighbour pair inside one lattice
    P->lattice = false;
    P->adj_dir.assign(P->adj_nbr.size(), -1);
    P->lats.clear();
    P->lat_maxnl = 0;
    if (nl->n_lat > 0 && nl->lat_desc) {
        P->lats.assign(nl->lat_desc, nl->lat_desc + 4 * nl->n_lat);
    } else if (nl->lat_nx > 0 && nl->lat_ny > 0 && nl->lat_nl > 0) {
        P->lats = {0, nl->lat_nx, nl->lat_ny, nl->lat_nl};
    }
    std::vector<int32_t> lat_of;   // caller id -> lattice
    bool ok = !P->lats.empty();
    if (ok) {
        lat_of.assign(n, -1);
        int64_t expect = 0;
        for (size_t k = 0; k < P->lats.size() / 4 && ok; ++k) {
            const int64_t off = P->lats[4 * k], nx = P->lats[4 * k + 1], ny = P->lats[4 * k + 2],
                          nz = P->lats[4 * k + 3];
            ok = off == expect && nx > 0 && ny > 0 && nz > 0 && nz <= 3 && off + nx * ny * nz <= n;
            if (ok) {
                for (int64_t q = off; q < off + nx * ny * nz; ++q) lat_of[q] = (int32_t)k;
                expect = off + nx * ny * nz;
                P->lat_maxnl = std::max<int32_t>(P->lat_maxnl, (int32_t)nz);
            }
        }
        ok = ok && expect == n;
    }
    for (int i = 0; i < n && ok; ++i) {
        const int L = lat_of[i];
        const int off = P->lats[4 * L], nx = P->lats[4 * L + 1], ny = P->lats[4 * L + 2];
        const int li = i - off;
        const int xi = li % nx, yi = (li / nx) % ny, zi = li / (nx * ny);
        for (int64_t k = P->adj_ptr[i]; k < P->adj_ptr[i + 1] && ok; ++k) {
            const int j = P->adj_nbr[k];
            if (lat_of[j] != L) { ok = false; break; }
            const int lj = j - off;
            const int dx = lj % nx - xi, dy = (lj / nx) % ny - yi, dz = lj / (nx * ny) - zi;
            if (dx == 1 && dy == 0 && dz == 0) P->adj_dir[k] = 0;
            else if (dx == 0 && dy == 1 && dz == 0) P->adj_dir[k] = 1;
            else if (dx == 0 && dy == 0 && dz == 1) P->adj_dir[k] = 2;
            else if (!((dx == -1 && dy == 0 && dz == 0) || (dx == 0 && dy == -1 && dz == 0) ||
                       (dx == 0 && dy == 0 && dz == -1))) ok = false;
        }
    }
    if (!ok) { P->lats.clear(); P->lat_maxnl = 0; }
    P->lattice = ok;

    // --- colouring: BFS 2-colouring (red-black), else greedy multicolour; a grid that
    // takes the lattice inner solve keeps its natural order (one colour)
    const bool natural = P->lattice && lattice_policy != INT32_MIN &&
                         (lattice_policy > 0 || (lattice_policy == 0 && auto_lattice_k(P->lat_maxnl, n) > 0));
    std::vector<int32_t> colour(n, natural ? 0 : -1);
    bool bipartite = !natural;
    if (!natural) {
        std::vector<int32_t> q; q.reserve(n);
        for (int s = 0; s < n && bipartite; ++s) {
            if (colour[s] >= 0) continue;
            colour[s] = 0; q.clear(); q.push_back(s);
            for (size_t h = 0; h < q.size() && bipartite; ++h) {
                int u = q[h];
                for (int64_t k = P->adj_ptr[u]; k < P->adj_ptr[u + 1]; ++k) {
                    int w = P->adj_nbr[k];
                    if (colour[w] < 0) { colour[w] = 1 - colour[u]; q.push_back(w); }
                    else if (colour[w] == colour[u]) { bipartite = false; break; }
                }
            }
        }
    }
    int ncol = natural ? 1 : 2;
    // four colours on a lattice: ((x + l) mod 2) + 2 (y mod 2) differs across every x, y and via
    // neighbour pair, so each class is independent; another valid Gauss-Seidel order
    const bool four = !natural && colouring == PG_COLOUR_FOUR && P->lattice;
    if (natural) {
        // one colour
    } else if (four) {
        for (size_t L = 0; L < P->lats.size() / 4; ++L) {
            const int32_t off = P->lats[4 * L], lnx = P->lats[4 * L + 1], lny = P->lats[4 * L + 2],
                          lnl = P->lats[4 * L + 3];
            for (int32_t l = 0; l < lnl; ++l)
                for (int32_t y = 0; y < lny; ++y)
                    for (int32_t x = 0; x < lnx; ++x)
                        colour[off + ((int64_t)l * lny + y) * lnx + x] = ((x + l) & 1) + 2 * (y & 1);
        }
        ncol = 0;
        for (int i = 0; i < n; ++i) ncol = std::max(ncol, colour[i] + 1);
        // a class no node fell into (a lattice one column or row wide) is dropped
        std::vector<int32_t> remap(4, -1);
        int m = 0;
        for (int c = 0; c < ncol; ++c)
            for (int i = 0; i < n; ++i)
                if (colour[i] == c) { remap[c] = m++; break; }
        for (int i = 0; i < n; ++i) colour[i] = remap[colour[i]];
        ncol = m;
    } else if (!bipartite || colouring == PG_COLOUR_FOUR) {
        std::fill(colour.begin(), colour.end(), -1);
        ncol = 0;
        bipartite = false;
        std::vector<int32_t> seen(kMaxColours + 1, -1);
        for (int i = 0; i < n; ++i) {
            for (int64_t k = P->adj_ptr[i]; k < P->adj_ptr[i + 1]; ++k) {
                int c = colour[P->adj_nbr[k]];
                if (c >= 0 && c <= kMaxColours) seen[c] = i;
            }
            int c = 0;
            while (c <= kMaxColours && seen[c] == i) ++c;
            if (c >= kMaxColours)
                return fail(PG_ERR_UNSUPPORTED, "graph needs more than 16 colours for the parallel update");
            colour[i] = c; ncol = std::max(ncol, c + 1);
        }
    } else {
        bool any1 = false;
        for (int i = 0; i < n; ++i) any1 |= colour[i] == 1;
        if (!any1) ncol = 1;
    }
    P->ncol = ncol;

    // --- permutation: colour-major, caller order inside a colour, each colour padded to kSlice
    std::vector<int32_t> ccount(ncol, 0);
    for (int i = 0; i < n; ++i) ccount[colour[i]]++;
    P->colour_start[0] = 0;
    for (int c = 0; c < ncol; ++c)
        P->colour_start[c + 1] = P->colour_start[c] + (ccount[c] + kSlice - 1) / kSlice * kSlice;
    for (int c = ncol + 1; c <= kMaxColours; ++c) P->colour_start[c] = P->colour_start[ncol];
    const int32_t np = P->colour_start[ncol];
    P->n_pad = np;
    P->perm.assign(n, -1);
    P->orig.assign(np, -1);
    {
        std::vector<int32_t> fillc(P->colour_start, P->colour_start + ncol);
        for (int i = 0; i < n; ++i) { int k = fillc[colour[i]]++; P->perm[i] = k; P->orig[k] = i; }
    }

    P->node_lat.assign(np, -1);
    if (P->lattice)
        for (int q = 0; q < np; ++q)
            if (P->orig[q] >= 0) P->node_lat[q] = lat_of[P->orig[q]];

    // --- SELL slices, diagonal-offset form where the slice's columns are constant offsets
    const int32_t nsl = np / kSlice;
    P->n_slices = nsl;
    P->slice_off.assign(nsl + 1, 0);
    P->slice_w.assign(nsl, 0);
    P->slice_doff.assign(nsl + 1, 0);
    P->dia_off.clear();
    P->n_dia_slices = 0;
    std::vector<std::vector<int32_t>> slice_offsets(nsl);
    std::vector<int32_t> uni;
    for (int s = 0; s < nsl; ++s) {
        int kmax = 0;
        uni.clear();
        for (int q = 0; q < kSlice; ++q) {
            int i = s * kSlice + q, o = P->orig[i];
            if (o < 0) continue;
            int64_t d = P->adj_ptr[o + 1] - P->adj_ptr[o];
            kmax = std::max<int>(kmax, (int)d);
            for (int64_t k = P->adj_ptr[o]; k < P->adj_ptr[o + 1]; ++k)
                uni.push_back(P->perm[P->adj_nbr[k]] - i);
        }
        std::sort(uni.begin(), uni.end());
        uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
        bool dia = !uni.empty() && (int)uni.size() <= kmax + 2 && (int)uni.size() <= 12;
        if (dia) {
            int lo = s * kSlice, hi = lo + kSlice - 1;
            if (lo + uni.front() < 0 || hi + uni.back() >= np) dia = false;
        }
        if (dia) {
            slice_offsets[s] = uni;
            P->slice_w[s] = (int)uni.size();
            P->n_dia_slices++;
        } else {
            P->slice_w[s] = kmax;
        }
        P->slice_off[s + 1] = P->slice_off[s] + (int64_t)P->slice_w[s] * kSlice;
        P->slice_doff[s + 1] = P->slice_doff[s] + (dia ? (int)uni.size() : 0);
        if (dia) P->dia_off.insert(P->dia_off.end(), uni.begin(), uni.end());
    }
    P->n_ell = P->slice_off[nsl];
    P->ell_col.assign(P->n_ell, 0);
    P->ell_adj.assign(P->n_ell, -1);
    for (int s = 0; s < nsl; ++s) {
        const int W = P->slice_w[s];
        const bool dia = P->slice_doff[s + 1] > P->slice_doff[s];
        for (int q = 0; q < kSlice; ++q) {
            int i = s * kSlice + q, o = P->orig[i];
            for (int k = 0; k < W; ++k) {
                int64_t e = P->slice_off[s] + (int64_t)k * kSlice + q;
                P->ell_col[e] = dia ? i + slice_offsets[s][k] : i;   // empty slot reads itself, weight 0
            }
            if (o < 0) continue;
            int k = 0;
            for (int64_t a = P->adj_ptr[o]; a < P->adj_ptr[o + 1]; ++a) {
                int j = P->perm[P->adj_nbr[a]];
                int slot;
                if (dia) {
                    slot = (int)(std::lower_bound(slice_offsets[s].begin(), slice_offsets[s].end(), j - i) -
                                 slice_offsets[s].begin());
                } else {
                    slot = k++;
                }
                int64_t e = P->slice_off[s] + (int64_t)slot * kSlice + q;
                P->ell_col[e] = j;
                P->ell_adj[e] = a;
            }
        }
    }

    // --- loads, per permuted node
    P->ld_ptr.assign(np + 1, 0);
    for (int64_t e = 0; e < nl->n_i; ++e) {
        if (nl->i_a[e] >= 0) P->ld_ptr[P->perm[nl->i_a[e]] + 1]++;
        if (nl->i_b[e] >= 0) P->ld_ptr[P->perm[nl->i_b[e]] + 1]++;
    }
    for (int i = 0; i < np; ++i) P->ld_ptr[i + 1] += P->ld_ptr[i];
    P->ld_idx.assign(P->ld_ptr[np], 0);
    {
        std::vector<int32_t> f(P->ld_ptr.begin(), P->ld_ptr.end() - 1);
        for (int64_t e = 0; e < nl->n_i; ++e) {
            if (nl->i_a[e] >= 0) P->ld_idx[f[P->perm[nl->i_a[e]]]++] = (int32_t)(e + 1);
            if (nl->i_b[e] >= 0) P->ld_idx[f[P->perm[nl->i_b[e]]]++] = -(int32_t)(e + 1);
        }
    }
    if (nl->n_i) {
        if (nl->i_ptr[nl->n_i] > (int64_t)INT32_MAX - 1) {   // the device indexes breakpoints in 32 bits
            *why = "too many PWL breakpoints (at most 2^31 - 2 in one netlist)";
            return PG_ERR_INVALID_ARG;
        }
        P->pwl_ptr.assign(nl->i_ptr, nl->i_ptr + nl->n_i + 1);
        P->pwl_t.assign(nl->i_t, nl->i_t + nl->i_ptr[nl->n_i]);
        P->pwl_v.assign(nl->i_v, nl->i_v + nl->i_ptr[nl->n_i]);
        pwl_aux(P->pwl_ptr, P->pwl_t, P->pwl_v, &P->pwl_s, &P->pwl_tk);
    } else {
        P->pwl_ptr.assign(1, 0); P->pwl_t.clear(); P->pwl_v.clear(); P->pwl_s.clear(); P->pwl_tk.clear();
    }

    // --- inductors
    P->n_l = (int32_t)nl->n_l;
    P->ind_a.resize(nl->n_l); P->ind_b.resize(nl->n_l); P->ind_invL.resize(nl->n_l);
    P->ind_ptr.assign(np + 1, 0);
    for (int64_t e = 0; e < nl->n_l; ++e) {
        int32_t a = nl->l_a[e], b = nl->l_b[e];
        P->ind_a[e] = a >= 0 ? P->perm[a] : a;
        P->ind_b[e] = b >= 0 ? P->perm[b] : b;
        P->ind_invL[e] = 1.0 / nl->l_val[e];
        if (a >= 0) P->ind_ptr[P->perm[a] + 1]++;
        if (b >= 0) P->ind_ptr[P->perm[b] + 1]++;
    }
    for (int i = 0; i < np; ++i) P->ind_ptr[i + 1] += P->ind_ptr[i];
    P->ind_idx.assign(P->ind_ptr[np], 0);
    {
        std::vector<int32_t> f(P->ind_ptr.begin(), P->ind_ptr.end() - 1);
        for (int64_t e = 0; e < nl->n_l; ++e) {
            if (nl->l_a[e] >= 0) P->ind_idx[f[P->perm[nl->l_a[e]]]++] = (int32_t)(e + 1);
            if (nl->l_b[e] >= 0) P->ind_idx[f[P->perm[nl->l_b[e]]]++] = -(int32_t)(e + 1);
        }
    }
    return PG_OK;
}

pg_status refill_values(const pg_netlist* nl, Packed* P, std::string* why) {
    auto fail = [&](const std::string& m) { if (why) *why = m; return PG_ERR_INVALID_ARG; };
    const int32_t n = P->n;
    std::fill(P->adj_g.begin(), P->adj_g.end(), 0.0);
    std::fill(P->adj_il.begin(), P->adj_il.end(), 0.0);
    P->g_gnd.assign(n, 0.0); P->il_gnd.assign(n, 0.0); P->cap.assign(n, 0.0);
    P->inj_g.assign(n, 0.0); P->inj_il.assign(n, 0.0);
    auto tv = [&](int32_t t) { return t == PG_GROUND ? 0.0 : nl->vdd[-2 - t]; };
    auto entry = [&](int32_t i, int32_t j) -> int64_t {
        const auto b = P->adj_nbr.begin() + P->adj_ptr[i], e = P->adj_nbr.begin() + P->adj_ptr[i + 1];
        const auto it = std::lower_bound(b, e, j);
        return (it != e && *it == j) ? (int64_t)(it - P->adj_nbr.begin()) : -1;
    };
    for (int64_t e = 0; e < nl->n_r; ++e) {
        const int32_t a = nl->r_a[e], b = nl->r_b[e];
        const double g = nl->r_g[e];
        if (!finite_pos(g)) return fail("resistor conductance must be > 0");
        if (a >= 0 && b >= 0) {
            P->adj_g[entry(a, b)] += g;
            P->adj_g[entry(b, a)] += g;
        } else if (a >= 0 || b >= 0) {
            const int32_t i = a >= 0 ? a : b, o = a >= 0 ? b : a;
            P->g_gnd[i] += g; P->inj_g[i] += g * tv(o);
        }
    }
    for (int64_t e = 0; e < nl->n_l; ++e) {
        const int32_t a = nl->l_a[e], b = nl->l_b[e];
        if (!finite_pos(nl->l_val[e])) return fail("inductance must be > 0");
        const double il = 1.0 / nl->l_val[e];
        P->ind_invL[e] = il;
        if (a >= 0 && b >= 0) {
            P->adj_il[entry(a, b)] += il;
            P->adj_il[entry(b, a)] += il;
        } else if (a >= 0 || b >= 0) {
            const int32_t i = a >= 0 ? a : b, o = a >= 0 ? b : a;
            P->il_gnd[i] += il; P->inj_il[i] += il * tv(o);
        }
    }
    for (int64_t e = 0; e < nl->n_c; ++e) {
        if (!finite_pos(nl->c_val[e])) return fail("capacitance must be > 0");
        const int32_t a = nl->c_a[e], b = nl->c_b[e];
        if (a >= 0 || b >= 0) P->cap[a >= 0 ? a : b] += nl->c_val[e];
    }
    return PG_OK;
}

}  // namespace pg
