// schedule.cpp -- host side of the aligned / contained decomposition
// (Sec. 2.2, Steps 1-4), emitted as flat work lists (see fm_sched.h).
#include <algorithm>
#include <vector>

#include "fm_internal.cuh"
#include "fm_sched.h"

namespace {

// Cut points of [0, len) where (off + x) crosses a multiple of T' = 2^lt.
void add_cuts(int64_t len, int64_t off, int lt, std::vector<int64_t>& pts)
{
    const int64_t T = (int64_t)1 << lt;
    int64_t first = ((off + T - 1) / T) * T - off;  // first x > =0 with (off+x) % T == 0
    if (first == 0) first = T;
    for (int64_t x = first; x < len; x += T) pts.push_back(x);
}

std::vector<int64_t> partition(int64_t len, const int64_t* offs, int n, int lt)
{
    std::vector<int64_t> pts = {0, len};
    for (int k = 0; k < n; ++k) add_cuts(len, offs[k], lt, pts);
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    return pts;
}

bool overlap(const fm_sub& x, const fm_sub& y)
{
    if (x.m.base != y.m.base) return false;
    if (x.rows == 0 || x.cols == 0 || y.rows == 0 || y.cols == 0) return false;
    return x.row0 < y.row0 + y.rows && y.row0 < x.row0 + x.rows && x.col0 < y.col0 + y.cols &&
           y.col0 < x.col0 + x.cols;
}

}  // namespace

int fm_check_matrix(const fm_matrix& m)
{
    if (m.log2_T < 0 || m.log2_T > 10 || m.log2_grid < 0) return FM_EINVAL;
    if (m.log2_T + m.log2_grid > 20) return FM_EINVAL;
    if (m.base == nullptr || ((uintptr_t)m.base & 15) != 0) return FM_EINVAL;
    return FM_OK;
}

int fm_check_sub(const fm_sub& s)
{
    int rc = fm_check_matrix(s.m);
    if (rc != FM_OK) return rc;
    const int64_t n = fm_side(s.m);
    if (s.rows < 0 || s.cols < 0 || s.row0 < 0 || s.col0 < 0) return FM_EINVAL;
    if (s.row0 + s.rows > n || s.col0 + s.cols > n) return FM_EINVAL;
    return FM_OK;
}

int fm_check_product(const fm_sub& C, const fm_sub& A, const fm_sub& B, bool same_tile)
{
    FM_TRY(fm_check_sub(C));
    FM_TRY(fm_check_sub(A));
    FM_TRY(fm_check_sub(B));
    if (A.rows != C.rows || B.cols != C.cols || A.cols != B.rows) return FM_EINVAL;
    if (same_tile && (A.m.log2_T != C.m.log2_T || B.m.log2_T != C.m.log2_T)) return FM_EINVAL;
    if (overlap(C, A) || overlap(C, B)) return FM_EINVAL;
    return FM_OK;
}

void fm_decompose_call(const fm_sub& C, const fm_sub& A, const fm_sub& B, int32_t call_index,
                       std::vector<FmWorkItem>& items, std::vector<FmLPiece>& lps,
                       int32_t* lp_begin, int32_t* lp_count)
{
    const int lt = C.m.log2_T;
    const int64_t T = (int64_t)1 << lt;
    const int64_t M = C.rows, N = C.cols, K = A.cols;
    *lp_begin = (int32_t)lps.size();
    *lp_count = 0;
    if (M == 0 || N == 0) return;

    // l: cut at A's tile-column and B's tile-row boundaries.
    if (K > 0) {
        const int64_t offs[2] = {A.col0, B.row0};
        std::vector<int64_t> lp = partition(K, offs, 2, lt);
        for (size_t t = 0; t + 1 < lp.size(); ++t) {
            const int64_t l0 = lp[t];
            FmLPiece q;
            q.a_tj = (int32_t)((A.col0 + l0) >> lt);
            q.a_c = (int32_t)((A.col0 + l0) & (T - 1));
            q.b_ti = (int32_t)((B.row0 + l0) >> lt);
            q.b_r = (int32_t)((B.row0 + l0) & (T - 1));
            q.len = (int32_t)(lp[t + 1] - l0);
            q.l0 = (int32_t)l0;
            lps.push_back(q);
        }
        *lp_count = (int32_t)(lp.size() - 1);
    }

    // Output parts: i cut at C's tile rows, j at C's tile columns.
    const int64_t coff_r[1] = {C.row0};
    const int64_t coff_c[1] = {C.col0};
    std::vector<int64_t> ip = partition(M, coff_r, 1, lt);
    std::vector<int64_t> jp = partition(N, coff_c, 1, lt);
    for (size_t a = 0; a + 1 < ip.size(); ++a) {
        const int64_t i0 = ip[a], rows = ip[a + 1] - ip[a];
        const int64_t ar = A.row0 + i0;
        const int64_t a_r = ar & (T - 1);
        const int64_t a_split = std::min<int64_t>(rows, T - a_r);
        for (size_t b = 0; b + 1 < jp.size(); ++b) {
            const int64_t j0 = jp[b], cols = jp[b + 1] - jp[b];
            const int64_t bc = B.col0 + j0;
            const int64_t b_c = bc & (T - 1);
            FmWorkItem w;
            w.call = call_index;
            w.c_ti = (int32_t)((C.row0 + i0) >> lt);
            w.c_tj = (int32_t)((C.col0 + j0) >> lt);
            w.c_r = (int32_t)((C.row0 + i0) & (T - 1));
            w.c_c = (int32_t)((C.col0 + j0) & (T - 1));
            w.rows = (int32_t)rows;
            w.cols = (int32_t)cols;
            w.a_ti = (int32_t)(ar >> lt);
            w.a_r = (int32_t)a_r;
            w.a_split = (int32_t)a_split;
            w.b_tj = (int32_t)(bc >> lt);
            w.b_c = (int32_t)b_c;
            w.b_split = (int32_t)std::min<int64_t>(cols, T - b_c);
            w.i0 = (int32_t)i0;
            w.j0 = (int32_t)j0;
            w.pad = 0;
            items.push_back(w);
        }
    }
}

extern "C" int64_t fm_decompose(fm_sub C, fm_sub A, fm_sub B, int64_t* out, int64_t cap)
{
    // Host-only: validate shapes (base pointers may be any non-null aligned value).
    int rc = fm_check_product(C, A, B, true);
    if (rc != FM_OK) return rc;
    std::vector<FmWorkItem> items;
    std::vector<FmLPiece> lps;
    int32_t b, n;
    fm_decompose_call(C, A, B, 0, items, lps, &b, &n);
    int64_t count = 0;
    for (const FmWorkItem& w : items) {
        const int64_t isplit[3] = {0, w.a_split, w.rows};
        const int64_t jsplit[3] = {0, w.b_split, w.cols};
        for (int32_t q = 0; q < n; ++q) {
            const FmLPiece& lp = lps[b + q];
            for (int si = 0; si < 2; ++si) {
                if (isplit[si] >= isplit[si + 1]) continue;
                for (int sj = 0; sj < 2; ++sj) {
                    if (jsplit[sj] >= jsplit[sj + 1]) continue;
                    if (count < cap && out) {
                        int64_t* o = out + 6 * count;
                        o[0] = w.i0 + isplit[si];
                        o[1] = w.i0 + isplit[si + 1];
                        o[2] = w.j0 + jsplit[sj];
                        o[3] = w.j0 + jsplit[sj + 1];
                        o[4] = lp.l0;
                        o[5] = lp.l0 + lp.len;
                    }
                    ++count;
                }
            }
        }
    }
    return count;
}
