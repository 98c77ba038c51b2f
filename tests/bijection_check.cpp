// Host check of the product's bijection arithmetic (csrc/bijection.cuh):
//   * the multiply-high quotient equals x / b for every b in [2, 256] and every
//     x < 256 b (all shapes of cells up to 65536 particles);
//   * for each request "n k0 k1 k2 k3 k4 k5" on stdin, prints a, b, then pi(r)
//     for r = 0..n-1 and the inverse at every position, for comparison with the
//     oracle's table by the Python test;
//   * the table-driven rounds (bij_enc_tab, bij_dec_tab, as the kernels run them)
//     give the same pi and inverse.
#include <cstdio>
#include "../paper_2508_06771_gb300/csrc/bijection.cuh"
using namespace ltpc;

int main() {
    for (uint32_t b = 2; b <= 256; ++b) {
        const uint32_t mb = 0xFFFFFFFFu / b + 1u;
        for (uint32_t x = 0; x < 256u * b; ++x)
            if (bij_umulhi(x, mb) != x / b) { std::printf("FAIL quotient b=%u x=%u\n", b, x); return 1; }
    }
    unsigned n, k[6];
    while (std::scanf("%u %u %u %u %u %u %u", &n, &k[0], &k[1], &k[2], &k[3], &k[4], &k[5]) == 7) {
        BijParams B;
        B.n = n;
        bij_shape(n, &B.a, &B.b, &B.mb);
        for (int i = 0; i < 6; ++i) B.key[i] = k[i];
        static unsigned char tab[6][256];
        for (int i = 0; i < 6; ++i) {
            const uint32_t m = (i & 1) ? B.b : B.a, lim = (i & 1) ? B.a : B.b;
            for (uint32_t r = 0; r < lim; ++r) tab[i][r] = (unsigned char)bij_round(r, B.key[i], m);
        }
        auto rt = [&](int i, uint32_t r) -> uint32_t { return tab[i][r]; };
        for (uint32_t r = 0; r < n; ++r) {
            uint32_t y = bij_enc_tab(B, rt, r);
            while (y >= n) y = bij_enc_tab(B, rt, y);
            uint32_t x = bij_dec_tab(B, rt, r);
            while (x >= n) x = bij_dec_tab(B, rt, x);
            if (y != bij_forward(B, r) || x != bij_inverse(B, r)) {
                std::printf("FAIL tables n=%u r=%u\n", n, r);
                return 1;
            }
        }
        std::printf("%u %u\n", B.a, B.b);
        for (uint32_t r = 0; r < n; ++r) std::printf("%u ", bij_forward(B, r));
        std::printf("\n");
        for (uint32_t q = 0; q < n; ++q) std::printf("%u ", bij_inverse(B, q));
        std::printf("\n");
    }
    std::printf("bijection arithmetic OK\n");
    return 0;
}
