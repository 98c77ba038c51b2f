// Exhaustive host check of the cell kernel's ownership arithmetic: every
// position, bucket and home item has exactly one owner, every owner's range
// fits its per-CTA capacity, and pair slots never straddle CTAs.
#include <cstdio>
#include <cstdlib>
#include "../paper_2508_06771_gb300/csrc/ltpc_index.h"
using namespace ltpc;

static int fail(const char* what, unsigned n, unsigned C, unsigned x) {
    std::printf("FAIL %s n=%u C=%u x=%u\n", what, n, C, x);
    return 1;
}

int main(int argc, char** argv) {
    unsigned nmax = argc > 1 ? (unsigned)std::atoi(argv[1]) : 70000;
    const unsigned Cs[] = {1, 2, 4, 8, 16};
    for (unsigned C : Cs) {
        for (unsigned n = 1; n <= nmax; n += (n < 3000 ? 1 : 61)) {
            unsigned capl = (n + C - 1) / C;           // smallest admissible per-CTA capacity
            if (capl & 1) capl += 1;
            if (n > cluster_capacity(C, capl)) return fail("capacity", n, C, capl);
            unsigned half = n_half(n), nb = n_buckets(n);
            unsigned prev_end = 0;
            for (unsigned r = 0; r < C; ++r) {
                unsigned b = pos_begin(r, n, C), e = pos_end(r, n, C);
                if (b != prev_end && !(b >= n && prev_end == n)) return fail("pos contiguity", n, C, r);
                if (b & 1) return fail("odd pos begin", n, C, r);
                if (e > b && e - b > capl) return fail("pos range > capl", n, C, r);
                prev_end = e > b ? e : prev_end;
                unsigned hb = split_begin(r, n, C), he = split_begin(r + 1, n, C);
                if (he - hb > capl) return fail("home > capl", n, C, r);
                unsigned bb = split_begin(r, nb, C), be = split_begin(r + 1, nb, C);
                if (be - bb > capl) return fail("buckets > capl", n, C, r);
            }
            if (prev_end != n) return fail("pos cover", n, C, prev_end);
            for (unsigned q = 0; q < n; ++q) {
                unsigned o = pos_owner(q, n, C);
                if (o >= C || q < pos_begin(o, n, C) || q >= pos_end(o, n, C)) return fail("pos owner", n, C, q);
                if ((q ^ 1u) < n && pos_owner(q ^ 1u, n, C) != o) return fail("pair straddles", n, C, q);
            }
            for (unsigned t = 0; t < nb; ++t) {
                unsigned o = split_owner(t, nb, C);
                if (o >= C || t < split_begin(o, nb, C) || t >= split_begin(o + 1, nb, C)) return fail("bucket owner", n, C, t);
            }
            (void)half;
        }
    }
    std::printf("index arithmetic OK\n");
    return 0;
}
