// Host-only consistency check of the plan-time table layout (run by
// tests/test_layouts.py on the CPU; no device call): the byte count the handle
// allocates for the linear-fold constants (fold_bytes) covers the layout the
// kernels address (FoldLayout + TileTables), for every state/measurement size
// the library instantiates, both precisions and tile counts up to 4096; and
// every table read by bulk copies or 16-byte loads starts on a 16-byte
// boundary.
#include <cstdio>
#include "../paper_2512_13319_gb300/csrc/handle.h"
#include "../paper_2512_13319_gb300/csrc/lti_fold.cuh"

template <int N, int M, typename S>
static int check()
{
    using TT = mapk::TileTables<N, M, S>;
    int bad = 0;
    for (long nt = 1; nt <= 4096; ++nt) {
        const size_t have = mapk::fold_bytes(N, M, sizeof(S), nt), need = TT::bytes(nt);
        const size_t offs[] = {TT::tl_off(), TT::p_off(), TT::f_off(nt), TT::pi_off(nt), TT::g_off(nt)};
        bool ok = need <= have;
        for (size_t o : offs) ok = ok && o % 16 == 0;
        // the transposed products are read with 16-byte loads only when a
        // matrix is a whole number of 16-byte words (load_run_aligned)
        if ((N * N) % (16 / (int)sizeof(S)) == 0) ok = ok && TT::qt_off(nt) % 16 == 0;
        if (!ok && bad++ < 3)
            std::printf("N=%d M=%d S=%zu nt=%ld: need %zu have %zu\n", N, M, sizeof(S), nt, need, have);
    }
    return bad;
}

int main()
{
    int bad = 0;
    bad += check<2, 1, float>() + check<2, 1, double>();
    bad += check<3, 1, float>() + check<3, 1, double>();
    bad += check<4, 2, float>() + check<4, 2, double>();
    bad += check<5, 2, float>() + check<5, 2, double>();
    bad += check<6, 3, float>() + check<6, 3, double>();
    std::printf(bad ? "FAIL %d\n" : "OK\n", bad);
    return bad ? 1 : 0;
}
