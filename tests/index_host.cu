// Host checks of index arithmetic the line-pass kernels rely on:
//  (1) j mod Ns by a multiply-high with the reciprocal set_stage_products
//      stores (ns_mag), against the % operator, for every product of radices
//      a schedule can reach below 4096 and every j < 4096;
//  (2) the split last-stage twiddle factors of the 2048- and 4096-point
//      schedules (p2_tw_split): the entries the kernel multiplies, taken from
//      the middle stage's table and the 16 x 15 factor table at the offsets
//      the kernel uses, give exp(-2 pi i k r / L) for every k and r;
//  (3) the XOR-swizzled first work generation of the strided power-of-two
//      passes (p2_swz0): one-to-one on a row, inside the row stride, and the
//      second stage's per-thread shortcut reads the same slots;
//  (4) the work-row strides: the 16 threads of a half-warp of a stage that
//      maps them across lines touch 16 different banks (8-byte words mod 16),
//      for the strided power-of-two passes and for every line length and
//      tile shape of the batched-uneven kernel, and its padded landing rows.
//  (5) the batched-uneven kernel's stage twiddles formed as powers (radix 8
//      from w and w^4, radix 4 and 5 from w and w^2) in FP32: within a few ulp.
// Prints one line per check: name, cases, failures (or worst error).
#include <cmath>
#include <complex>
#include <cstdio>
#include <vector>

#include "fft_p2.cuh"
#include "fft_uneven.cuh"

using namespace fbfft;
using cd = std::complex<double>;

static unsigned umulhi32(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }

static cd w(long long m, long long D) { return std::polar(1.0, -2.0 * M_PI * (double)(m % D) / (double)D); }

// 1 when the 8-byte words of one half-warp (n of them) fall on n different
// banks, or repeat a word (a broadcast), 0 otherwise.
static int banks_distinct(const long long* words, int n)
{
    long long seen[16];
    for (int b = 0; b < 16; ++b) seen[b] = -1;
    for (int i = 0; i < n; ++i) {
        const int b = (int)(words[i] & 15);
        if (seen[b] >= 0 && seen[b] != words[i]) return 0;
        seen[b] = words[i];
    }
    return 1;
}

int main()
{
    // (1) every 5-smooth Ns < 4096 as the product before a stage
    long long cases = 0, bad = 0;
    for (int a = 0; a < 12; ++a)
        for (int b = 0; b < 8; ++b)
            for (int c = 0; c < 6; ++c) {
                const long long ns = (1LL << a) * (long long)std::pow(3, b) * (long long)std::pow(5, c);
                if (ns < 2 || ns >= 4096) continue;
                PassDesc d{};
                d.nst = 2;
                d.radix[0] = (int)ns;  // stage 1 then sees Ns = ns
                d.radix[1] = 2;
                set_stage_products(d);
                if (d.ns[1] != ns) ++bad;
                for (unsigned j = 0; j < 4096; ++j) {
                    const unsigned k = j - umulhi32(j, d.ns_mag[1]) * (unsigned)ns;
                    ++cases;
                    if (k != j % ns) ++bad;
                }
            }
    std::printf("mod_by_reciprocal %lld %lld\n", cases, bad);

    // (2) split twiddles of the last stage
    for (int lg = 9; lg <= 12; ++lg) {
        if (!p2_tw_split(lg)) {
            std::printf("split_lg%d none 0\n", lg);
            continue;
        }
        const long long L = 1LL << lg;
        const int ns1 = pow2_ns(lg, 1), ns2 = pow2_ns(lg, 2), r1 = pow2_radix(lg, 1), r2 = pow2_radix(lg, 2);
        // shared-memory image: stage-1 table at p2_tws_off(lg, 1) ([r-1][k], D = ns1 * r1),
        // factor table at p2_tws_off(lg, 2) ([r-1][kl], D = L), as the twiddle jobs define them
        const int total = p2_smem_twiddles(lg);
        cd* tws = new cd[total];
        for (int r = 1; r < r1; ++r)
            for (int k = 0; k < ns1; ++k) tws[p2_tws_off(lg, 1) + (r - 1) * ns1 + k] = w((long long)r * k, (long long)ns1 * r1);
        for (int r = 1; r < 16; ++r)
            for (int kl = 0; kl < 16; ++kl) tws[p2_tws_off(lg, 2) + (r - 1) * 16 + kl] = w((long long)r * kl, L);
        double worst = 0;
        long long n = 0;
        for (int k = 0; k < ns2; ++k)
            for (int r = 1; r < r2; ++r) {
                const cd got = tws[p2_tws_off(lg, 1) + (k >> 4) + (r - 1) * ns1] * tws[p2_tws_off(lg, 2) + (k & 15) + (r - 1) * 16];
                const cd want = w((long long)k * r, (long long)ns2 * r2);
                worst = std::fmax(worst, std::abs(got - want));
                ++n;
            }
        const bool sizes_ok = ns2 * r2 == L && ns2 == 16 * ns1 && p2_tws_off(lg, 2) + 16 * 15 == total;
        std::printf("split_lg%d %lld %.3e %d\n", lg, n, worst, sizes_ok ? 1 : 0);
        // the kernel's arithmetic in FP32: table entries rounded to float, the
        // factors for r = 1 and 8 as table products, the others stepped by one
        // complex multiply each (the kernel's cmul)
        double worst_step = 0;
        long long ns_ = 0;
        auto f2 = [](cd z) { return make_float2((float)z.real(), (float)z.imag()); };
        for (int k = 0; k < ns2; ++k) {
            const float2 th0 = f2(tws[p2_tws_off(lg, 1) + (k >> 4)]), tl0 = f2(tws[p2_tws_off(lg, 2) + (k & 15)]);
            const float2 th7 = f2(tws[p2_tws_off(lg, 1) + (k >> 4) + 7 * ns1]);
            const float2 tl7 = f2(tws[p2_tws_off(lg, 2) + (k & 15) + 7 * 16]);
            const float2 w1 = cmul(th0, tl0), w8 = cmul(th7, tl7);
            float2 wr = w1;
            for (int r = 1; r < 16; ++r) {
                if (r == 8) wr = w8;
                else if (r > 1) wr = cmul(wr, w1);
                const cd want = w((long long)k * r, (long long)ns2 * r2);
                worst_step = std::fmax(worst_step, std::abs(cd(wr.x, wr.y) - want));
                ++ns_;
            }
        }
        std::printf("split_step_lg%d %lld %.3e\n", lg, ns_, worst_step);
        delete[] tws;
    }

    // (3) swizzled first generation
    {
        long long n = 0, bad = 0, configs = 0;
        const int ios[2] = {kIoCC, kIoCCP};
        for (int threads : {256, 512})
            for (int lg = 9; lg <= 11; ++lg)
                for (int io : ios) {
                    if (!p2_swz0(threads, lg, io)) continue;
                    ++configs;
                    const int L = 1 << lg, LS = p2_work_stride(threads, lg, io);
                    const int LR1 = L / pow2_radix(lg, 1);
                    std::vector<char> used(LS, 0);
                    for (int i = 0; i < L; ++i) {
                        const int x = spad_x(i);
                        ++n;
                        if (x < 0 || x >= LS || used[x]) ++bad;
                        else used[x] = 1;
                    }
                    for (int j = 0; j < LR1; ++j)
                        for (int r = 0; r < 16; ++r) {
                            ++n;
                            if (spad_x(j + r * LR1) != spad((j ^ ((j >> 2) & 3)) + r * LR1)) ++bad;
                        }
                }
        std::printf("swizzle %lld %lld %lld\n", n, bad, configs);
    }

    // (4a) strided power-of-two passes: the last stage reads the work rows
    // across lines (t fastest), positions j + r L/R
    {
        long long n = 0, bad = 0;
        const int ios[3] = {kIoCC, kIoCCP, kIoNC};
        for (int threads : {256, 512})
            for (int lg = 7; lg <= 12; ++lg)
                for (int io : ios) {
                    const int T = p2_tile_lines(threads, lg, io);
                    if (T > 16 || pow2_nst(lg) < 2) continue;
                    const int L = 1 << lg, LS = p2_work_stride(threads, lg, io);
                    const int R = pow2_radix(lg, pow2_nst(lg) - 1), LR = L / R, H = 16 / T;
                    for (int j0 = 0; j0 < LR; j0 += H)
                        for (int r = 0; r < R; ++r) {
                            long long wd[16];
                            int m = 0;
                            for (int t = 0; t < T; ++t)
                                for (int h = 0; h < H && j0 + h < LR; ++h) wd[m++] = (long long)t * LS + spad(j0 + h + r * LR);
                            ++n;
                            if (!banks_distinct(wd, m)) ++bad;
                        }
                }
        std::printf("p2_rows %lld %lld\n", n, bad);
    }

    // (4b) batched-uneven kernel: every 5-smooth L <= 2048, every tile shape
    // the planner can pick; work rows for lines-fast and positions-fast
    // stages, padded landing rows for the first stage of contiguous tiles
    {
        long long n = 0, bad = 0, land = 0, land_bad = 0;
        for (int L = 1; L <= kUnevenCap; ++L) {
            int x = L;
            for (int p : {2, 3, 5})
                while (x % p == 0) x /= p;
            if (x != 1) continue;
            for (int cf = 0; cf < 2; ++cf)
                for (long long T = 1; T * L <= kUnevenCap && T <= (cf ? 32 : kUnevenThreads); T *= 2) {
                    const int LS = uneven_line_stride(L, T, cf != 0);
                    if (LS < L) ++bad;
                    const long long G = kUnevenThreads / T;
                    if (cf && T <= 16) {  // lines fast: T lines x 16/T positions
                        const int H = (int)(16 / T);
                        for (int j0 = 0; j0 + H <= L; j0 += H) {
                            long long wd[16];
                            int m = 0;
                            for (int t = 0; t < T; ++t)
                                for (int h = 0; h < H; ++h) wd[m++] = (long long)t * LS + j0 + h;
                            ++n;
                            if (!banks_distinct(wd, m)) ++bad;
                        }
                    }
                    if (!cf && G < 16) {  // positions fast: 16/G lines x G positions
                        for (int j0 = 0; j0 + G <= L; j0 += (int)G) {
                            long long wd[16];
                            int m = 0;
                            for (long long t = 0; t < 16 / G; ++t)
                                for (long long h = 0; h < G; ++h) wd[m++] = t * LS + j0 + h;
                            ++n;
                            if (!banks_distinct(wd, m)) ++bad;
                        }
                    }
                    const int lr = uneven_land_row(L, T, false);
                    if (T >= 2 && T <= 8) {
                        ++land;
                        const int H = (int)(16 / T);
                        if (lr < L || (lr & 1)) ++land_bad;
                        for (int j0 = 0; j0 + H <= L; j0 += H) {
                            long long wd[16];
                            int m = 0;
                            for (int t = 0; t < T; ++t)
                                for (int h = 0; h < H; ++h) wd[m++] = (long long)t * lr + j0 + h;
                            if (!banks_distinct(wd, m)) ++land_bad;
                        }
                    } else if (lr != 0) {
                        ++land_bad;
                    }
                }
        }
        std::printf("uneven_rows %lld %lld\n", n, bad);
        std::printf("uneven_land %lld %lld\n", land, land_bad);
    }

    // (5) stage twiddles of the batched-uneven kernel by powers: for a
    // butterfly with k < Ns of a radix-R stage the factors are w^r, w =
    // w_{Ns R}^k; radix 8 takes w and w^4 from the table (rounded to FP32)
    // and forms w^2 = w w, w^3 = w^2 w, w^5 = w^4 w, w^6 = w^4 w^2, w^7 = w^4 w^3,
    // radix 4 and 5 take w and w^2 and form w^3 = w^2 w (and w^4 = w^2 w^2),
    // all with the kernel's FP32 cmul: every 5-smooth Ns with Ns R <= 2048
    {
        auto f2 = [](cd z) { return make_float2((float)z.real(), (float)z.imag()); };
        double worst = 0;
        long long n = 0;
        for (int R : {8, 4, 5})
            for (long long Ns = 1; Ns * R <= 2048; ++Ns) {
                long long m = Ns;
                for (long long p : {2LL, 3LL, 5LL})
                    while (m % p == 0) m /= p;
                if (m != 1) continue;
                const long long D = Ns * R;
                for (long long k = 0; k < Ns; ++k) {
                    float2 f[8];
                    f[1] = f2(w(k, D));
                    if (R == 8) {
                        f[4] = f2(w(4 * k, D));
                        f[2] = cmul(f[1], f[1]);
                        f[3] = cmul(f[2], f[1]);
                        f[5] = cmul(f[4], f[1]);
                        f[6] = cmul(f[4], f[2]);
                        f[7] = cmul(f[4], f[3]);
                    } else {
                        f[2] = f2(w(2 * k, D));
                        f[3] = cmul(f[2], f[1]);
                        f[4] = cmul(f[2], f[2]);
                    }
                    for (int r = 1; r < R; ++r) {
                        worst = std::fmax(worst, std::abs(cd(f[r].x, f[r].y) - w(k * r, D)));
                        ++n;
                    }
                }
            }
        std::printf("uneven_step %lld %.3e\n", n, worst);
    }
    return 0;
}
