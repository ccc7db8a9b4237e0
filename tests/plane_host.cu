// Host emulation of the plane pass (fft_plane.cuh): every CTA of a cluster,
// every compute thread, each phase between two barriers run to completion
// before the next, with the kernel's own index functions and butterflies.
// Checks that every shared-memory slot, owner CTA and row a thread touches is
// in range, that no two threads write one slot in a phase, and that the
// result equals the 2-D DFT (row then column sums of exp(s 2 pi i n k / L),
// in double).  Prints "plane L1 L2 threads dir worst_rel_l2 violations" per
// case, and per shape "banks L1 L2 threads" followed by the worst bank
// conflict degree of each phase's shared-memory accesses (1 = none).
#include <cmath>
#include <complex>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <random>
#include <vector>

#include "fft_plane.cuh"

using namespace fbfft;
using cd = std::complex<double>;

template <int LG1, int LG2, int TH, bool FWD>
static void run_case(unsigned seed, int* violations, double* rel)
{
    using P = PlaneCfg<LG1, LG2, TH>;
    constexpr int L1 = P::L1, L2 = P::L2, CS = P::CS, T = P::THREADS;
    std::mt19937 rng(seed);
    std::uniform_real_distribution<float> U(-1.f, 1.f);
    std::vector<float2> x(L1 * L2);
    for (auto& e : x) e = make_float2(U(rng), U(rng));
    // stage-1 tables as the twiddle jobs define them: entry (r-1)*16 + k = exp(-2 pi i r k / L)
    auto table = [](int L, int R) {
        std::vector<float2> t(16 * (R - 1));
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < 16; ++k) {
                const double a = -2.0 * M_PI * (double)((r * k) % L) / (double)L;
                t[(r - 1) * 16 + k] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
        return t;
    };
    const std::vector<float2> twr = table(L2, P::G2), twc = table(L1, P::G1);
    const float nanv = std::nanf("");
    std::vector<std::vector<float2>> buf(CS, std::vector<float2>(P::BUF, make_float2(nanv, nanv)));
    int bad = 0;
    auto slot_ok = [&](int s) {
        if (s < 0 || s >= P::BUF) {
            ++bad;
            return false;
        }
        return true;
    };
    std::vector<int> mark(P::BUF);
    auto phase_begin = [&] { std::fill(mark.begin(), mark.end(), 0); };
    auto write = [&](std::vector<float2>& b, int s, float2 v) {
        if (!slot_ok(s)) return;
        if (mark[s]++) ++bad;  // two writes of one slot in one phase
        b[s] = v;
    };
    // load: rows [q R1, (q+1) R1), dense at stride RS
    for (int q = 0; q < CS; ++q)
        for (int r = 0; r < P::R1; ++r)
            for (int c = 0; c < L2; ++c) buf[q][r * P::RS + c] = x[(q * P::R1 + r) * L2 + c];
    for (int q = 0; q < CS; ++q) {
        // row stage 0: all reads, barrier, all writes
        std::vector<float2> v((size_t)T * 16);
        for (int t = 0; t < T; ++t) {
            const int row = P::row_of(t), j0 = P::rj_of(t);
            if (row < 0 || row >= P::R1) ++bad;
            for (int r = 0; r < 16; ++r) {
                const int s = row * P::RS + P::row_s0_in(j0, r);
                v[t * 16 + r] = slot_ok(s) ? buf[q][s] : make_float2(0, 0);
            }
        }
        phase_begin();
        for (int t = 0; t < T; ++t) {
            dft<16, FWD>(&v[t * 16]);
            for (int r = 0; r < 16; ++r)
                write(buf[q], P::row_of(t) * P::RS + P::row_s0_out(P::rj_of(t), r), v[t * 16 + r]);
        }
        // row stage 1, in place (each butterfly reads and writes its own slots)
        phase_begin();
        for (int t = 0; t < T; ++t) {
            const int row = P::row_of(t), j0 = P::rj_of(t);
            for (int u = 0; u < 16 / P::G2; ++u) {
                const int j = j0 + P::G2 * u;
                float2 w[P::G2];
                for (int r = 0; r < P::G2; ++r) {
                    const int s = row * P::RS + P::row_s1(j, r);
                    w[r] = slot_ok(s) ? buf[q][s] : make_float2(0, 0);
                }
                for (int r = 1; r < P::G2; ++r) w[r] = twmul<FWD>(w[r], twr[(r - 1) * 16 + j]);
                dft<P::G2, FWD>(w);
                for (int r = 0; r < P::G2; ++r) write(buf[q], row * P::RS + P::row_s1(j, r), w[r]);
            }
        }
    }
    // column gather from every CTA (cluster barrier), then every CTA's writes
    std::vector<std::vector<float2>> g(CS, std::vector<float2>((size_t)T * 16));
    for (int q = 0; q < CS; ++q)
        for (int t = 0; t < T; ++t) {
            const int cl = P::cl_of(t), cj = P::cj_of(t);
            if (cj < 0 || cj >= P::G1 || cl < 0 || cl >= P::W) ++bad;
            const int c = q * P::W + cl;
            for (int r = 0; r < 16; ++r) {
                const int o = P::owner(r), lr = P::lrow(cj, r);
                // the row this input must be: j + G1 r of the plane
                if (o < 0 || o >= CS || lr < 0 || lr >= P::R1 || o * P::R1 + lr != cj + P::G1 * r) {
                    ++bad;
                    continue;
                }
                const int s = lr * P::RS + P::col_slot(c);
                g[q][t * 16 + r] = slot_ok(s) ? buf[o][s] : make_float2(0, 0);
            }
        }
    for (int q = 0; q < CS; ++q) {
        phase_begin();
        for (int t = 0; t < T; ++t) {
            const int cl = P::cl_of(t), cj = P::cj_of(t);
            dft<16, FWD>(&g[q][t * 16]);
            for (int r = 0; r < 16; ++r) write(buf[q], P::blk(16 * cj + r, cl), g[q][t * 16 + r]);
        }
        phase_begin();
        for (int t = 0; t < T; ++t) {
            const int cl = P::cl_of(t), cj = P::cj_of(t);
            for (int u = 0; u < 16 / P::G1; ++u) {
                const int j = cj + P::G1 * u;
                float2 w[P::G1];
                for (int r = 0; r < P::G1; ++r) {
                    const int s = P::blk(j + 16 * r, cl);
                    w[r] = slot_ok(s) ? buf[q][s] : make_float2(0, 0);
                }
                for (int r = 1; r < P::G1; ++r) w[r] = twmul<FWD>(w[r], twc[(r - 1) * 16 + j]);
                dft<P::G1, FWD>(w);
                for (int r = 0; r < P::G1; ++r) write(buf[q], P::blk(j + 16 * r, cl), w[r]);
            }
        }
    }
    // store: CTA q's column block -> columns [q W, (q+1) W)
    std::vector<cd> y((size_t)L1 * L2);
    for (int q = 0; q < CS; ++q)
        for (int m = 0; m < L1; ++m)
            for (int c = 0; c < P::W; ++c) {
                const float2 e = buf[q][m * P::W + c];
                y[(size_t)m * L2 + q * P::W + c] = cd(e.x, e.y);
            }
    // reference: DFT of every row, then of every column, in double
    const double sgn = FWD ? -1.0 : 1.0;
    std::vector<cd> a((size_t)L1 * L2), ref((size_t)L1 * L2);
    for (int n1 = 0; n1 < L1; ++n1)
        for (int k2 = 0; k2 < L2; ++k2) {
            cd s = 0;
            for (int n2 = 0; n2 < L2; ++n2)
                s += cd(x[n1 * L2 + n2].x, x[n1 * L2 + n2].y) *
                     std::polar(1.0, sgn * 2.0 * M_PI * (double)((n2 * k2) % L2) / L2);
            a[(size_t)n1 * L2 + k2] = s;
        }
    for (int k2 = 0; k2 < L2; ++k2)
        for (int k1 = 0; k1 < L1; ++k1) {
            cd s = 0;
            for (int n1 = 0; n1 < L1; ++n1)
                s += a[(size_t)n1 * L2 + k2] * std::polar(1.0, sgn * 2.0 * M_PI * (double)((n1 * k1) % L1) / L1);
            ref[(size_t)k1 * L2 + k2] = s;
        }
    double num = 0, den = 0;
    for (size_t i = 0; i < y.size(); ++i) {
        num += std::norm(y[i] - ref[i]);
        den += std::norm(ref[i]);
    }
    *rel = std::sqrt(num / den);
    if (!(*rel == *rel)) *rel = 1e30;  // NaN: a slot was read before it was written
    *violations = bad;
}

// Shared-memory bank conflicts of the kernel's accesses: for every phase and
// every value r a thread moves, each half-warp's 16 eight-byte slots (the
// unit one conflict-free wavefront serves) must fall in 16 different slot
// positions mod 16; identical slots are one broadcast.  Returns the worst
// number of distinct slots sharing a position, per phase.
template <int LG1, int LG2, int TH>
static void bank_check()
{
    using P = PlaneCfg<LG1, LG2, TH>;
    auto worst = [](auto slot_of) {
        int w = 1;
        for (int t0 = 0; t0 < P::THREADS; t0 += 16)
            for (int r = 0; r < 16; ++r) {
                int cnt[16] = {0};
                int seen[16];
                int ns = 0;
                for (int l = 0; l < 16; ++l) {
                    const int s = slot_of(t0 + l, r);
                    if (s < 0) continue;
                    bool dup = false;
                    for (int k = 0; k < ns; ++k) dup = dup || seen[k] == s;
                    if (dup) continue;
                    seen[ns++] = s;
                    w = std::max(w, ++cnt[s & 15]);
                }
            }
        return w;
    };
    const int row_in = worst([](int t, int r) { return P::row_of(t) * P::RS + P::row_s0_in(P::rj_of(t), r); });
    const int row_out = worst([](int t, int r) { return P::row_of(t) * P::RS + P::row_s0_out(P::rj_of(t), r); });
    const int row_s1 = worst([](int t, int r) {
        const int u = r / P::G2, rr = r % P::G2;  // the thread's 16 values: butterfly u, input rr
        return P::row_of(t) * P::RS + P::row_s1(P::rj_of(t) + P::G2 * u, rr);
    });
    const int gather = worst([](int t, int r) {
        return P::lrow(P::cj_of(t), r) * P::RS + P::col_slot(P::cl_of(t));  // CTA 0's columns
    });
    const int col_out = worst([](int t, int r) { return P::blk(16 * P::cj_of(t) + r, P::cl_of(t)); });
    const int col_s1 = worst([](int t, int r) {
        const int u = r / P::G1, rr = r % P::G1;
        return P::blk(P::cj_of(t) + P::G1 * u + 16 * rr, P::cl_of(t));
    });
    std::printf("banks %d %d %d %d %d %d %d %d %d\n", 1 << LG1, 1 << LG2, TH, row_in, row_out, row_s1, gather, col_out,
                col_s1);
}

template <int LG1, int LG2, int TH>
static void both(unsigned seed)
{
    bank_check<LG1, LG2, TH>();
    int v;
    double e;
    run_case<LG1, LG2, TH, true>(seed, &v, &e);
    std::printf("plane %d %d %d fwd %.3e %d\n", 1 << LG1, 1 << LG2, TH, e, v);
    run_case<LG1, LG2, TH, false>(seed + 1, &v, &e);
    std::printf("plane %d %d %d inv %.3e %d\n", 1 << LG1, 1 << LG2, TH, e, v);
}

int main()
{
    both<8, 7, 512>(11);
    both<7, 7, 512>(12);
    both<8, 8, 512>(13);
    both<7, 8, 512>(14);
    both<8, 7, 256>(15);
    both<7, 7, 256>(16);
    both<7, 8, 256>(17);
    return 0;
}
