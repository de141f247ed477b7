// Brickwall layout and window-pass planner (host code).
//
// The sweep over K gates is split into "window passes": a pass picks a
// window S of w neighbouring qubits and applies, to every tile of 2^w
// amplitudes that share the other n - w qubit values, every not-yet-applied
// gate that lies inside S and whose predecessors are applied. A pass is one
// read and one write of the states in HBM, however many gates it holds; the
// gates themselves run out of shared memory. The backward sweep runs the same
// passes in reverse order, each gate in reverse order.
//
// Between passes the qubit -> address-bit layout is permuted inside the
// current window so that the lowest kLowBits address bits always hold qubits
// of both the current and the next window: every tile then reads and writes
// runs of at least 2^kLowBits contiguous amplitudes.
#include <algorithm>
#include <cmath>

#include "../../include/hvp.h"
#include "internal.h"

namespace hvp {

int num_gates(int n, int L) {
    if (n < 2 || L < 1) return -1;
    int k = 0;
    for (int layer = 1; layer <= L; ++layer) k += (n - (layer - 1) % 2) / 2;
    return k;
}

// Sec. 3.1 / Fig. computational-passes: layer l (1-based) has offset
// (l-1) mod 2 and gates on (i, i+1) for i = offset, offset + 2, ...
void brickwall_layout(int n, int L, std::vector<int>& fq) {
    fq.clear();
    for (int layer = 1; layer <= L; ++layer)
        for (int i = (layer - 1) % 2; i + 1 <= n - 1; i += 2) fq.push_back(i);
}

// Shared-memory bit order of a window: qubits q0, q2, q4 first so that no gate
// (which acts on neighbouring qubits) has both bits among index bits 0..2.
static std::vector<int> smem_order(const std::vector<int>& asc) {
    std::vector<int> out;
    for (size_t t = 0; t < asc.size() && t <= 4; t += 2) out.push_back(asc[t]);
    for (int q : asc)
        if (std::find(out.begin(), out.end(), q) == out.end()) out.push_back(q);
    return out;
}

struct Window { int lo, hi; };  // qubits [lo, hi]

static bool in_window(const Window& w, int q) { return q >= w.lo && q <= w.hi; }

// Greedy simulation of a window sequence; returns the passes as (window,
// gates). A window with nothing to do is dropped unless the windows before
// and after it share fewer than b qubits: then it stays as a transit pass
// (no gates, only the layout permutation) so that every consecutive pair of
// passes keeps b common qubits for the low address bits.
static int overlap(const Window& a, const Window& c) {
    return std::max(0, std::min(a.hi, c.hi) - std::max(a.lo, c.lo) + 1);
}

static bool simulate(int K, int b, const std::vector<int>& fq, const std::vector<int>& p1,
                     const std::vector<int>& p2, const std::vector<Window>& wins,
                     const std::vector<int>& seq_cycle,
                     std::vector<std::pair<int, std::vector<int>>>& out) {
    std::vector<char> done(K, 0);
    int ndone = 0, empty_run = 0;
    size_t pos = 0;
    std::vector<std::pair<int, std::vector<int>>> raw;
    while (ndone < K) {
        int wi = seq_cycle[pos % seq_cycle.size()];
        ++pos;
        std::vector<int> list;
        for (int g = 0; g < K; ++g) {
            if (done[g]) continue;
            if (!in_window(wins[wi], fq[g]) || !in_window(wins[wi], fq[g] + 1)) continue;
            if ((p1[g] >= 0 && !done[p1[g]]) || (p2[g] >= 0 && !done[p2[g]])) continue;
            done[g] = 1;
            ++ndone;
            list.push_back(g);
        }
        if (list.empty()) {
            if (++empty_run > 2 * (int)seq_cycle.size()) return false;
        } else {
            empty_run = 0;
        }
        raw.emplace_back(wi, std::move(list));
    }
    // Keep the passes with gates; between two passes whose windows share
    // fewer than b qubits insert the windows that lie between them along the
    // chain (windows are sorted and neighbours share >= b qubits).
    out.clear();
    for (auto& pr : raw) {
        if (pr.second.empty()) continue;
        if (!out.empty() && overlap(wins[out.back().first], wins[pr.first]) < b) {
            int a = out.back().first, c = pr.first, step = c > a ? 1 : -1;
            for (int t = a + step; t != c; t += step) out.emplace_back(t, std::vector<int>());
        }
        out.push_back(std::move(pr));
    }
    return true;
}

// Beam search over window positions. A step moves to a window [lo, lo+w-1]
// that shares >= b qubits with the current one and applies every gate that
// is ready inside it (none: a transit pass). The cost of a plan is its
// number of passes, a step with more than kMaxGatesPerPass gates counting as
// several. Each step keeps the `width` cheapest partial plans (most gates
// applied first among equal costs), one per (applied set, window).
static bool beam_plan(int n, int w, int b, const std::vector<int>& fq, const std::vector<int>& p1,
                      const std::vector<int>& p2, std::vector<std::pair<Window, std::vector<int>>>& out) {
    const int K = (int)fq.size();
    const int nw = n - w + 1;
    const size_t width = 64;
    struct Node {
        int cost = 0, ndone = 0, lo = 0;
        std::vector<char> done;
        std::vector<std::pair<int, std::vector<int>>> hist;
    };
    auto step = [&](const Node& from, int lo, Node& to) {
        to.done = from.done;
        to.hist = from.hist;
        std::vector<int> list;
        for (int g = 0; g < K; ++g) {
            if (to.done[g] || fq[g] < lo || fq[g] + 1 > lo + w - 1) continue;
            if ((p1[g] >= 0 && !to.done[p1[g]]) || (p2[g] >= 0 && !to.done[p2[g]])) continue;
            to.done[g] = 1;
            list.push_back(g);
        }
        const int c = (int)list.size();
        to.cost = from.cost + (c == 0 ? 1 : (c + kMaxGatesPerPass - 1) / kMaxGatesPerPass);
        to.ndone = from.ndone + c;
        to.lo = lo;
        to.hist.emplace_back(lo, std::move(list));
    };
    auto better = [](const Node& x, const Node& y) {
        return x.cost != y.cost ? x.cost < y.cost : x.ndone > y.ndone;
    };
    std::vector<Node> cur;
    Node root;
    root.done.assign(K, 0);
    for (int lo = 0; lo < nw; ++lo) {
        Node nd;
        step(root, lo, nd);
        if (nd.ndone > 0) cur.push_back(std::move(nd));
    }
    bool found = false;
    Node best;
    for (int it = 0; it < 8 * K + 8 && !cur.empty(); ++it) {
        std::vector<Node> next;
        for (const Node& nd : cur) {
            if (nd.ndone == K) {
                if (!found || nd.cost < best.cost) { best = nd; found = true; }
                continue;
            }
            if (found && nd.cost + 1 >= best.cost) continue;
            for (int lo = 0; lo < nw; ++lo) {
                if (lo == nd.lo || overlap({nd.lo, nd.lo + w - 1}, {lo, lo + w - 1}) < b) continue;
                Node nx;
                step(nd, lo, nx);
                next.push_back(std::move(nx));
            }
        }
        std::sort(next.begin(), next.end(), better);
        cur.clear();
        std::vector<std::pair<int, std::vector<char>>> seen;
        for (Node& nd : next) {
            if (cur.size() >= width) break;
            bool dup = false;
            for (const auto& sv : seen)
                if (sv.first == nd.lo && sv.second == nd.done) { dup = true; break; }
            if (dup) continue;
            seen.emplace_back(nd.lo, nd.done);
            cur.push_back(std::move(nd));
        }
    }
    if (!found) return false;
    out.clear();
    for (auto& h : best.hist) out.emplace_back(Window{h.first, h.first + w - 1}, std::move(h.second));
    return true;
}

static int passes_after_split(const std::vector<std::pair<Window, std::vector<int>>>& v) {
    int P = 0;
    for (const auto& pr : v)
        P += pr.second.empty() ? 1 : (int)((pr.second.size() + kMaxGatesPerPass - 1) / kMaxGatesPerPass);
    return P;
}

int make_plan(int n, int L, int w, int b, Plan& plan) {
    if (n < 2 || n > kMaxN || L < 1 || w < 2 || w > kMaxW || b < 1 || b >= w) return HVP_EINVAL;
    plan = Plan();
    plan.n = n; plan.L = L; plan.w = std::min(w, n); plan.b = b;
    brickwall_layout(n, L, plan.first_qubit);
    const std::vector<int>& fq = plan.first_qubit;
    const int K = (int)fq.size();
    plan.K = K;
    std::vector<int> last(n, -1), p1(K), p2(K);
    for (int k = 0; k < K; ++k) {
        p1[k] = last[fq[k]];
        p2[k] = last[fq[k] + 1];
        last[fq[k]] = last[fq[k] + 1] = k;
    }

    std::vector<Window> wins;
    std::vector<std::pair<Window, std::vector<int>>> best;
    if (n <= w) {
        std::vector<int> all(K);
        for (int k = 0; k < K; ++k) all[k] = k;
        best.emplace_back(Window{0, n - 1}, all);
    } else {
        const int m = (n - b + (w - b) - 1) / (w - b);  // windows with overlaps >= b
        for (int j = 0; j < m; ++j) {
            int lo = (int)std::lround((double)j * (n - w) / (double)(m - 1));
            wins.push_back({lo, lo + w - 1});
        }
        // Candidate window sequences: zig-zag and cyclic, from either end.
        std::vector<std::vector<int>> seqs;
        std::vector<int> fwd, zz;
        for (int j = 0; j < m; ++j) fwd.push_back(j);
        zz = fwd;
        for (int j = m - 2; j >= 1; --j) zz.push_back(j);
        std::vector<int> rfwd(fwd.rbegin(), fwd.rend()), rzz;
        for (int j : zz) rzz.push_back(m - 1 - j);
        seqs = {zz, fwd, rzz, rfwd};
        bool ok = false;
        for (auto& s : seqs) {
            std::vector<std::pair<int, std::vector<int>>> cand;
            if (!simulate(K, b, fq, p1, p2, wins, s, cand)) continue;
            std::vector<std::pair<Window, std::vector<int>>> cw;
            for (auto& pr : cand) cw.emplace_back(wins[pr.first], std::move(pr.second));
            if (!ok || passes_after_split(cw) < passes_after_split(best)) { best = std::move(cw); ok = true; }
        }
        std::vector<std::pair<Window, std::vector<int>>> bw;
        if (beam_plan(n, w, b, fq, p1, p2, bw) && (!ok || passes_after_split(bw) < passes_after_split(best))) {
            best = std::move(bw);
            ok = true;
        }
        if (!ok) return HVP_EINVAL;
    }

    // Split passes over the shared-memory gate budget (a prefix of a valid
    // pass order is itself valid).
    std::vector<std::pair<Window, std::vector<int>>> split;
    for (auto& pr : best) {
        if (pr.second.empty()) split.push_back(pr);
        for (size_t s = 0; s < pr.second.size(); s += kMaxGatesPerPass) {
            size_t e = std::min(pr.second.size(), s + (size_t)kMaxGatesPerPass);
            split.emplace_back(pr.first, std::vector<int>(pr.second.begin() + s, pr.second.begin() + e));
        }
    }
    const int P = (int)split.size();
    plan.pass_of_gate.assign(K, -1);

    // Layouts. Order of qubits inside a window for the output: qubits shared
    // with the next window first (they land on the lowest address bits).
    auto window_qubits = [&](int p) {
        std::vector<int> q;
        for (int x = split[p].first.lo; x <= split[p].first.hi; ++x) q.push_back(x);
        return q;
    };
    auto ordered_for_next = [&](int p) {
        std::vector<int> cur = window_qubits(p), first, rest;
        if (p + 1 < P) {
            const Window& nx = split[p + 1].first;
            for (int q : cur) (in_window(nx, q) ? first : rest).push_back(q);
        } else {
            first = cur;
        }
        first.insert(first.end(), rest.begin(), rest.end());
        return first;
    };
    std::vector<int> pos(n, -1);
    if (n <= w) {
        for (int q = 0; q < n; ++q) pos[q] = n - 1 - q;   // standard layout
    } else {
        std::vector<int> order = ordered_for_next(0);
        std::vector<char> used(n, 0);
        int bit = 0;
        for (int q : order) { pos[q] = bit++; used[q] = 1; }
        for (int q = 0; q < n; ++q)
            if (!used[q]) pos[q] = bit++;
    }
    for (int p = 0; p < P; ++p) {
        PassPlan pp;
        std::vector<int> wq = window_qubits(p);
        pp.S = smem_order(wq);
        pp.gates = split[p].second;
        for (int g : pp.gates) plan.pass_of_gate[g] = p;
        pp.pos_in = pos;
        if (n > w && p + 1 < P && split[p + 1].first.lo != split[p].first.lo) {
            std::vector<int> B;
            for (int q : wq) B.push_back(pos[q]);
            std::sort(B.begin(), B.end());
            std::vector<int> order = ordered_for_next(p);
            for (size_t t = 0; t < order.size(); ++t) pos[order[t]] = B[t];
        }
        pp.pos_out = pos;
        plan.passes.push_back(std::move(pp));
    }
    // Every pass must keep address bits [0, b) local (checked, not assumed).
    for (auto& pp : plan.passes) {
        for (int bit = 0; bit < std::min(b, n); ++bit) {
            bool in_in = false, in_out = false;
            for (int q : pp.S) { in_in |= pp.pos_in[q] == bit; in_out |= pp.pos_out[q] == bit; }
            if (n > w && (!in_in || !in_out)) return HVP_EINVAL;
        }
    }
    return HVP_OK;
}

void build_dev_passes(const Plan& plan, std::vector<DevPass>& dps, std::vector<DevGate>& dgs) {
    dps.clear();
    dgs.clear();
    const int n = plan.n;
    for (const PassPlan& pp : plan.passes) {
        DevPass d{};
        const int w = (int)pp.S.size();
        d.w = w;
        d.nq = w;
        d.ng = n - w;
        d.n_gates = (int)pp.gates.size();
        d.gate_off = (int)dgs.size();
        std::vector<int> B;
        for (int q : pp.S) B.push_back(pp.pos_in[q]);
        std::sort(B.begin(), B.end());
        std::vector<int> q_at_in(n), q_at_out(n);
        for (int q = 0; q < n; ++q) { q_at_in[pp.pos_in[q]] = q; q_at_out[pp.pos_out[q]] = q; }
        auto jbit = [&](int q) { return (int)(std::find(pp.S.begin(), pp.S.end(), q) - pp.S.begin()); };
        for (int j = 0; j < w; ++j) d.sq[j] = pp.S[j];
        int r = 0;
        for (int bit = 0; bit < n; ++bit)
            if (!std::binary_search(B.begin(), B.end(), bit)) { d.gpos[r] = bit; d.gq[r] = q_at_in[bit]; ++r; }
        for (int x = 0; x < 64; ++x) {
            uint32_t off = 0, li = 0, lo = 0;
            for (int t = 0; t < 6 && t < w; ++t)
                if ((x >> t) & 1) {
                    off |= 1u << B[t];
                    li |= 1u << jbit(q_at_in[B[t]]);
                    lo |= 1u << jbit(q_at_out[B[t]]);
                }
            d.off_lo[x] = off; d.in_lo[x] = (uint16_t)li; d.out_lo[x] = (uint16_t)lo;
        }
        for (int y = 0; y < 256; ++y) {
            uint32_t off = 0, li = 0, lo = 0;
            for (int t = 6; t < w && t < 14; ++t)
                if ((y >> (t - 6)) & 1) {
                    off |= 1u << B[t];
                    li |= 1u << jbit(q_at_in[B[t]]);
                    lo |= 1u << jbit(q_at_out[B[t]]);
                }
            d.off_hi[y] = off; d.in_hi[y] = (uint16_t)li; d.out_hi[y] = (uint16_t)lo;
        }
        for (int g : pp.gates) {
            DevGate dg{};
            dg.k = g;
            dg.u = jbit(plan.first_qubit[g]);
            dg.v = jbit(plan.first_qubit[g] + 1);
            dgs.push_back(dg);
        }
        dps.push_back(d);
    }
}

}  // namespace hvp

extern "C" int hvp_num_gates(int n, int n_layers) { return hvp::num_gates(n, n_layers); }

extern "C" int hvp_plan_brickwall(int n, int n_layers, int window, int low_bits, int* pass_of_gate) {
    hvp::Plan plan;
    int rc = hvp::make_plan(n, n_layers, window, low_bits, plan);
    if (rc != HVP_OK) return rc;
    if (pass_of_gate)
        for (int k = 0; k < plan.K; ++k) pass_of_gate[k] = plan.pass_of_gate[k];
    return (int)plan.passes.size();
}
