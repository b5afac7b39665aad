// Prints the host-side weight constants of the CUDA path as hex floats, so that
// a test can check their exact sums in rational arithmetic: the stencil weights
// of Eq. 2.36 (make_stencil), the linear coefficients of the momentum-form
// equilibrium (LinearCoef), and the folded relaxation of Eq. 2.52 (make_relax).
// Host code only: it needs no GPU.
#include <cstdio>
#include <cstdlib>

#include "packed.cuh"

using namespace fdlbm;

int main(int argc, char **argv)
{
    const int n = argc > 1 ? std::atoi(argv[1]) : 101;
    for (int k = 0; k < n; ++k) {
        const double beta = (double)k / (n - 1);
        const Stencil<float> f = make_stencil<float>(beta);
        const Stencil<double> d = make_stencil<double>(beta);
        std::printf("stencil %.17g f %a %a %a %a d %a %a %a %a\n", beta, (double)f.wm1, (double)f.w0,
                    (double)f.w1, (double)f.w2, d.wm1, d.w0, d.w1, d.w2);
    }
    std::printf("linear f %a %a d %a %a\n", (double)LinearCoef<float>::c1, (double)LinearCoef<float>::c2,
                LinearCoef<double>::c1, LinearCoef<double>::c2);
    for (int k = 1; k < n; ++k) {
        const float b = (float)((double)k / n);
        const packed::RelaxK r = packed::make_relax(b);
        std::printf("relax %a %a %a %a %a %a %a %a %a\n", (double)b, (double)r.bw0.x, (double)r.bw1.x,
                    (double)r.bw2.x, (double)r.bc1.x, (double)r.bc2.x, (double)r.nbc1.x, (double)r.nbc2.x,
                    (double)r.omb.x);
    }
    return 0;
}
