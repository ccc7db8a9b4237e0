// Host check of the line-pass butterflies (dft<R, FWD> in fft_device.cuh)
// against the DFT sum written out in double: prints the largest relative
// error per (R, direction) over random inputs.
#include <cmath>
#include <cstdio>
#include <random>

#include "fft_device.cuh"

using namespace fbfft;

template <int R, bool FWD>
double check(std::mt19937& g)
{
    std::uniform_real_distribution<float> u(-1.f, 1.f);
    double worst = 0;
    for (int trial = 0; trial < 200; ++trial) {
        float2 v[R];
        double xr[R], xi[R];
        for (int n = 0; n < R; ++n) {
            v[n] = make_float2(u(g), u(g));
            xr[n] = v[n].x, xi[n] = v[n].y;
        }
        dft<R, FWD>(v);
        const double s = FWD ? -1.0 : 1.0;
        double num = 0, den = 0;
        for (int k = 0; k < R; ++k) {
            double yr = 0, yi = 0;
            for (int n = 0; n < R; ++n) {
                const double a = s * 2.0 * M_PI * (double)((n * k) % R) / R;
                yr += xr[n] * std::cos(a) - xi[n] * std::sin(a);
                yi += xr[n] * std::sin(a) + xi[n] * std::cos(a);
            }
            num += (v[k].x - yr) * (v[k].x - yr) + (v[k].y - yi) * (v[k].y - yi);
            den += yr * yr + yi * yi;
        }
        worst = std::fmax(worst, std::sqrt(num / den));
    }
    return worst;
}

template <int R>
void both(std::mt19937& g)
{
    printf("%d %.3e %.3e\n", R, check<R, true>(g), check<R, false>(g));
}

int main()
{
    std::mt19937 g(9);
    both<2>(g);
    both<3>(g);
    both<4>(g);
    both<5>(g);
    both<8>(g);
    both<16>(g);
    return 0;
}
