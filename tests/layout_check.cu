// Host-only consistency check of the plan-time table layout (run by
// tests/test_layouts.py on the CPU; no device call): the byte count the handle
// allocates for the linear-fold constants (fold_bytes) covers the layout the
// kernels address (FoldLayout + TileTables), for every state/measurement size
// the library instantiates, both precisions and tile counts up to 4096; and
// every table read by bulk copies or 16-byte loads starts on a 16-byte
// boundary.
#include <cstdio>
#include <vector>
#include "../paper_2512_13319_gb300/csrc/handle.h"
#include "../paper_2512_13319_gb300/csrc/lti_fold.cuh"
#include "../paper_2512_13319_gb300/csrc/scan.cuh"

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

// Shared memory of the single-launch solve: every area that a bulk copy
// writes or reads (observations, Gamma_i, level constants, co table, staged
// states) starts on a 16-byte boundary and the mbarriers on an 8-byte one,
// for every tile size and steps per thread.
template <int N, int M, typename S>
static int check_fused()
{
    using FS = mapk::FusedSmem<N, M, S>;
    int bad = 0;
    for (int B = 32; B <= 128; B *= 2)
        for (int K = 1; K <= 64; ++K) {
            const size_t w = sizeof(S);
            bool ok = FS::ys(B) * w % 16 == 0 && FS::gam(B, K) * w % 16 == 0 && FS::lv(B, K) * w % 16 == 0 &&
                      FS::co(B, K) * w % 16 == 0 && FS::bar(B, K) * w % 8 == 0 && FS::stage(B) * w % 16 == 0 &&
                      FS::bytes(B, K) >= (size_t)FS::end(B, K) * w;
            if (!ok && bad++ < 3) std::printf("fused N=%d M=%d S=%zu B=%d K=%d\n", N, M, w, B, K);
        }
    return bad;
}

// The product table's row index pi_index(nt, a, b) (row a holding b = a..nt-1)
// and the transposes' qt_index(b, a) (row b holding a = 0..b) each number the
// nt (nt + 1) / 2 pairs a <= b once, rows contiguous.
static int check_product_indices()
{
    using TT = mapk::TileTables<4, 2, float>;
    int bad = 0;
    for (long nt = 1; nt <= TT::PI_TILES; nt += (nt < 40 ? 1 : 37)) {
        const long tri = nt * (nt + 1) / 2;
        std::vector<int> seen_pi(tri, 0), seen_qt(tri, 0);
        long expect_pi = 0;
        for (long a = 0; a < nt; ++a)
            for (long b = a; b < nt; ++b) {
                const long i = TT::pi_index(nt, a, b);
                if (i != expect_pi++ || i < 0 || i >= tri) { ++bad; continue; }
                ++seen_pi[i];
            }
        for (long b = 0; b < nt; ++b)
            for (long a = 0; a <= b; ++a) {
                const long i = TT::qt_index(b, a);
                if (i < 0 || i >= tri || (a > 0 && i != TT::qt_index(b, a - 1) + 1)) { ++bad; continue; }
                ++seen_qt[i];
            }
        for (long i = 0; i < tri; ++i) bad += (seen_pi[i] != 1) + (seen_qt[i] != 1);
    }
    if (bad) std::printf("product indices: %d bad\n", bad);
    return bad;
}

// The right-child coefficient table co_p by tree level (lti_co_level): entry
// i = p >> (d + 1) of level d, p = (2i + 1) 2^d, component q at q * cnt + i
// with cnt = B >> (d + 1); the B - 1 entries of 4 N^2 components fill the
// 4 N^2 (B - 1) scalars once.
template <int N>
static int check_co_levels()
{
    int bad = 0;
    for (int B = 2; B <= 128; B *= 2) {
        const int total = 4 * N * N * (B - 1);
        std::vector<int> seen(total, 0);
        for (int p = 1; p < B; ++p) {
            const int d = __builtin_ctz(p), i = p >> (d + 1), cnt = B >> (d + 1);
            for (int q = 0; q < 4 * N * N; ++q) {
                const int o = mapk::lti_co_level<N>(B, d) + q * cnt + i;
                if (o < 0 || o >= total) { ++bad; continue; }
                ++seen[o];
            }
        }
        for (int o = 0; o < total; ++o) bad += seen[o] != 1;
    }
    if (bad) std::printf("co levels N=%d: %d bad\n", N, bad);
    return bad;
}

int main()
{
    int fb = check_product_indices();
    fb += check_co_levels<2>() + check_co_levels<3>() + check_co_levels<4>() + check_co_levels<5>() +
          check_co_levels<6>();
    fb += check_fused<2, 1, float>() + check_fused<2, 1, double>();
    fb += check_fused<3, 1, float>() + check_fused<3, 1, double>();
    fb += check_fused<4, 2, float>() + check_fused<4, 2, double>();
    fb += check_fused<5, 2, float>() + check_fused<5, 2, double>();
    fb += check_fused<6, 3, float>() + check_fused<6, 3, double>();
    int bad = 0;
    bad += check<2, 1, float>() + check<2, 1, double>();
    bad += check<3, 1, float>() + check<3, 1, double>();
    bad += check<4, 2, float>() + check<4, 2, double>();
    bad += check<5, 2, float>() + check<5, 2, double>();
    bad += check<6, 3, float>() + check<6, 3, double>();
    bad += fb;
    std::printf(bad ? "FAIL %d\n" : "OK\n", bad);
    return bad ? 1 : 0;
}
