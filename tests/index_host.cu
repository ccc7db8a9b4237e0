// Host checks of index arithmetic the line-pass kernels rely on:
//  (1) j mod Ns by a multiply-high with the reciprocal set_stage_products
//      stores (ns_mag), against the % operator, for every product of radices
//      a schedule can reach below 4096 and every j < 4096;
//  (2) the split last-stage twiddle factors of the 2048- and 4096-point
//      schedules (p2_tw_split): the entries the kernel multiplies, taken from
//      the middle stage's table and the 16 x 15 factor table at the offsets
//      the kernel uses, give exp(-2 pi i k r / L) for every k and r.
// Prints one line per check: name, cases, failures (or worst error).
#include <cmath>
#include <complex>
#include <cstdio>

#include "fft_p2.cuh"

using namespace fbfft;
using cd = std::complex<double>;

static unsigned umulhi32(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }

static cd w(long long m, long long D) { return std::polar(1.0, -2.0 * M_PI * (double)(m % D) / (double)D); }

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
        delete[] tws;
    }
    return 0;
}
