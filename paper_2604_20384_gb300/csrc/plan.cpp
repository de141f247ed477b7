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

// Shared-memory bit order chosen per pass for conflict-free tile loads and
// stores as well as gates. With 16-byte elements and the swizzle swz(),
// shared-memory index bit 0, 1, 2 moves an element across 16-byte bank
// groups 1, 2, 4, bits 3 and 4 both across 7, higher bits not at all. A
// phase of 8 threads touches 8 elements that differ in three index bits; they
// avoid each other's bank groups when those bits' images are linearly
// independent over GF(2). Gates vary the three lowest index bits outside
// their own two, which are independent as long as no gate has both qubits
// among bits 0..2 (the triple there is pairwise non-adjacent). Tile loads and
// stores visit elements in global order, so their phases vary three of the
// six lowest global address bits of the window (the thread order inside a
// 64-element block is chosen later, in choose_io_order). This picks the triple
// for bits 0..2 and the two qubits for bits 3, 4 so that some three of those
// six global bits have independent images both in the input and in the
// output layout of the pass; ties keep the fixed order.
static int gf2_rank3(int a, int b, int c) {
    int v[3] = {a, b, c}, r = 0;
    for (int bit = 2; bit >= 0; --bit) {
        int piv = -1;
        for (int i = r; i < 3; ++i)
            if ((v[i] >> bit) & 1) { piv = i; break; }
        if (piv < 0) continue;
        std::swap(v[r], v[piv]);
        for (int i = 0; i < 3; ++i)
            if (i != r && ((v[i] >> bit) & 1)) v[i] ^= v[r];
        ++r;
    }
    return r;
}

static std::vector<int> io_aware_smem_order(const std::vector<int>& wq, const std::vector<int>& pos_in,
                                            const std::vector<int>& pos_out) {
    const std::vector<int> dflt = smem_order(wq);
    const int w = (int)wq.size();
    if (w < 6) return dflt;
    std::vector<int> B;
    for (int q : wq) B.push_back(pos_in[q]);
    std::sort(B.begin(), B.end());
    int qin[6], qout[6];
    for (int b = 0; b < 6; ++b)
        for (int q : wq) {
            if (pos_in[q] == B[b]) qin[b] = q;
            if (pos_out[q] == B[b]) qout[b] = q;
        }
    auto cost_of = [&](const std::vector<int>& S) {
        auto img = [&](int q) {
            for (int i = 0; i < 5; ++i)
                if (S[i] == q) return i < 3 ? 1 << i : 7;
            return 0;
        };
        int best = 1 << 30;
        for (int e0 = 0; e0 < 6; ++e0)
            for (int e1 = e0 + 1; e1 < 6; ++e1)
                for (int e2 = e1 + 1; e2 < 6; ++e2) {
                    const int ri = gf2_rank3(img(qin[e0]), img(qin[e1]), img(qin[e2]));
                    const int ro = gf2_rank3(img(qout[e0]), img(qout[e1]), img(qout[e2]));
                    best = std::min(best, (1 << (3 - ri)) + (1 << (3 - ro)));
                }
        return best;
    };
    std::vector<int> best = dflt;
    int best_cost = cost_of(dflt);
    for (int a = 0; a < w && best_cost > 2; ++a)
        for (int b = a + 2; b < w; ++b)
            for (int c = b + 2; c < w; ++c)
                for (int x = 0; x < w; ++x)
                    for (int y = x + 1; y < w; ++y) {
                        if (x == a || x == b || x == c || y == a || y == b || y == c) continue;
                        std::vector<int> S = {wq[a], wq[b], wq[c], wq[x], wq[y]};
                        for (int q : wq)
                            if (std::find(S.begin(), S.end(), q) == S.end()) S.push_back(q);
                        const int cst = cost_of(S);
                        if (cst < best_cost) { best_cost = cst; best = S; }
                    }
    return best;
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
        pp.S = io_aware_smem_order(wq, pp.pos_in, pp.pos_out);
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

// Shared-memory wavefronts of one tile's load (SMEM slots from the lo/hi
// tables `slo`, `shi`) when thread t handles tile element perm(t mod 64) +
// 64 (t / 64): 16-byte accesses are served in phases of 8 lanes, and a phase
// takes as many wavefronts as the largest number of its lanes that fall in
// the same 16-byte bank group.
static long tile_io_wavefronts(const uint16_t* slo, const uint16_t* shi, int w, const int* perm) {
    const int Lt = 1 << w;
    long total = 0;
    for (int base = 0; base < Lt; base += 8) {
        int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < 8; ++i) {
            const int t = base + i;
            const int m = perm[t & 63] | (t & ~63);
            const unsigned l = slo[m & 63] | shi[m >> 6];
            ++cnt[swz(l) & 7];
        }
        total += *std::max_element(cnt, cnt + 8);
    }
    return total;
}

// Per pass, the order in which the threads of a CTA visit the elements of a
// 64-element block during tile loads and stores: the permutation of the six
// low element-index bits that minimises the shared-memory wavefronts of the
// load (input layout) plus the store (output layout). Element pairs stay in
// one 32-byte global sector (index bit 0 comes from a lane bit), so global
// accesses remain fully used sectors.
static void choose_io_order(DevPass& d, int w) {
    if (w < 6) return;
    int bits[6] = {0, 1, 2, 3, 4, 5};
    int best_perm[64];
    long best = -1;
    do {
        if (bits[0] == 5) continue;                      // bit 0 of the element index from a lane bit
        int perm[64];
        for (int x = 0; x < 64; ++x) {
            int m = 0;
            for (int b = 0; b < 6; ++b)
                if ((x >> bits[b]) & 1) m |= 1 << b;     // element bit b <- thread bit bits[b]
            perm[x] = m;
        }
        const long c = tile_io_wavefronts(d.in_lo, d.in_hi, w, perm) + tile_io_wavefronts(d.out_lo, d.out_hi, w, perm);
        if (best < 0 || c < best) {
            best = c;
            std::copy(perm, perm + 64, best_perm);
        }
    } while (std::next_permutation(bits, bits + 6));
    uint32_t off[64];
    uint16_t li[64], lo[64];
    for (int x = 0; x < 64; ++x) {
        off[x] = d.off_lo[best_perm[x]];
        li[x] = d.in_lo[best_perm[x]];
        lo[x] = d.out_lo[best_perm[x]];
    }
    std::copy(off, off + 64, d.off_lo);
    std::copy(li, li + 64, d.in_lo);
    std::copy(lo, lo + 64, d.out_lo);
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
        choose_io_order(d, w);
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

// Fused-block plan of the tensor-core schedule: the gate sequence split into
// blocks of kBlockQ neighbouring qubits [a, a + kBlockQ); a block holds every
// gate inside its qubits whose predecessors lie in earlier blocks or earlier
// in the same block, in circuit order. The beam search of the window planner
// (windows of kBlockQ qubits, no overlap condition between consecutive
// windows) minimises the number of blocks, i.e. of dense 2^kBlockQ x
// 2^kBlockQ products per amplitude.
int make_block_plan(int n, int L, std::vector<BlockPlan>& blocks) {
    blocks.clear();
    if (n < kBlockQ || n > kMaxN || L < 1) return HVP_EINVAL;
    std::vector<int> fq;
    brickwall_layout(n, L, fq);
    const int K = (int)fq.size();
    std::vector<int> last(n, -1), p1(K), p2(K);
    for (int k = 0; k < K; ++k) {
        p1[k] = last[fq[k]];
        p2[k] = last[fq[k] + 1];
        last[fq[k]] = last[fq[k] + 1] = k;
    }
    std::vector<std::pair<Window, std::vector<int>>> bw;
    if (n == kBlockQ) {
        std::vector<int> all(K);
        for (int k = 0; k < K; ++k) all[k] = k;
        bw.emplace_back(Window{0, n - 1}, all);
    } else if (!beam_plan(n, kBlockQ, 0, fq, p1, p2, bw)) {
        return HVP_EINVAL;
    }
    int covered = 0;
    for (auto& pr : bw) {
        if (pr.second.empty()) continue;
        covered += (int)pr.second.size();
        blocks.push_back(BlockPlan{pr.first.lo, std::move(pr.second)});
    }
    return covered == K ? HVP_OK : HVP_EINVAL;
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

// Block plan of the tensor-core schedule for tests: block_of_gate[k] = block
// of gate k, block_qubit[j] = first qubit of block j (arrays of K entries).
extern "C" int hvp_plan_blocks(int n, int n_layers, int* block_of_gate, int* block_qubit) {
    std::vector<hvp::BlockPlan> blocks;
    int rc = hvp::make_block_plan(n, n_layers, blocks);
    if (rc != HVP_OK) return rc;
    for (size_t j = 0; j < blocks.size(); ++j) {
        if (block_qubit) block_qubit[j] = blocks[j].a;
        if (block_of_gate)
            for (int k : blocks[j].gates) block_of_gate[k] = (int)j;
    }
    return (int)blocks.size();
}
