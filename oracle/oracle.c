/*
 * oracle.c -- plain, slow, FP64 CPU reference of the TreeCode method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  The CUDA library never
 * includes, links or calls it, and this file uses nothing from the CUDA path.
 *
 * What it computes (Sec. 2 of the paper, plus the canonical tree readings
 * stated in each function):
 *   orc_direct        Eq. 1, direct particle-particle (PP) summation with
 *                     Plummer softening; potential -G m / sqrt(r^2+eps^2).
 *   orc_box           root box: lo = min, L = smallest power of two > extent.
 *   orc_keys          21-bit quantisation per axis, 63-bit Morton interleave.
 *   orc_sort          order by (key, original index).
 *   orc_octree        octree of Sec. 2 (space split into octants, recursively,
 *                     down to single-particle cells), generalised to a leaf
 *                     capacity, numbered breadth first.
 *   orc_moments       mass, centre of mass and traceless quadrupole per cell
 *                     (Sec. 2: far groups act through their total mass at the
 *                     centre of mass; the quadrupole is the next term).
 *   orc_groups        walk groups: key-order chunks, cut at coarse jumps.
 *   orc_lists         group walk with the theta opening criterion (Sec. 2).
 *   orc_tree_forces   cell expansion for accepted cells + exact PP sum for the
 *                     near leaves, self term excluded (Eq. 1).
 * Compiled with -O2 -ffp-contract=off (no FMA contraction, no fast-math),
 * following the strict-IEEE build setting of Sec. 3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BITS 21
#define ORC_MAXLEVEL 21

/* ------------------------------------------------------------------------ */
/* Eq. 1: a_i = sum_{j != i} G m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
 * phi_i = - sum_{j != i} G m_j / sqrt(|r_j - r_i|^2 + eps^2).
 * x is (3, n) structure of arrays; a is (3, nt); targets are indices into x.
 * Each target's sum runs over j in ascending order. */
void orc_direct(int64_t n, const double *x, const double *m, double G, double eps,
                int64_t nt, const int64_t *tgt, double *a, double *phi)
{
    const double *X = x, *Y = x + n, *Z = x + 2 * n;
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = tgt[t];
        double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            double r = sqrt(r2);
            double w = G * m[j] / (r2 * r);
            ax += w * dx; ay += w * dy; az += w * dz;
            p -= G * m[j] / r;
        }
        a[t] = ax; a[nt + t] = ay; a[2 * nt + t] = az;
        if (phi) phi[t] = p;
    }
}

/* ------------------------------------------------------------------------ */
/* Root box.  lo_d = min_i x_id, hi_d = max_i x_id, ext = max_d (hi_d - lo_d),
 * L = 2^k the smallest power of two with L > ext (L = 1 when ext = 0).
 * Returns 0, or -1 when a coordinate is NaN or infinite, or -2 when n < 1. */
int orc_box(int64_t n, const double *x, double *lo, int32_t *k_out)
{
    if (n < 1) return -2;
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        double mn = x[d * n], mx = x[d * n];
        for (int64_t i = 0; i < n; ++i) {
            double v = x[d * n + i];
            if (!isfinite(v)) return -1;
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        lo[d] = mn;
        if (mx - mn > ext) ext = mx - mn;
    }
    int32_t k = 0;
    if (ext > 0.0) {
        double L = 1.0;
        if (ext >= L) {
            while (!(L > ext)) { L *= 2.0; ++k; }
        } else {
            while (L * 0.5 > ext) { L *= 0.5; --k; }
        }
    }
    *k_out = k;
    return 0;
}

/* Quantisation q_d = min(2^21 - 1, floor((x_d - lo_d) * 2^(21-k))) -- one
 * rounding, in the subtraction -- and the key whose bit 3b+2 is bit b of q_x,
 * bit 3b+1 is bit b of q_y and bit 3b is bit b of q_z (b = 0..20). */
void orc_keys(int64_t n, const double *x, const double *lo, int32_t k,
              uint32_t *q, uint64_t *key)
{
    const double scale = ldexp(1.0, ORC_BITS - k);
    const double qmax = (double)((1u << ORC_BITS) - 1u);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t qq[3];
        for (int d = 0; d < 3; ++d) {
            double diff = x[d * n + i] - lo[d];
            double s = floor(diff * scale);
            if (s > qmax) s = qmax;
            if (s < 0.0) s = 0.0;
            qq[d] = (uint32_t)s;
            if (q) q[d * n + i] = qq[d];
        }
        uint64_t kk = 0;
        for (int b = 0; b < ORC_BITS; ++b) {
            kk |= (uint64_t)((qq[0] >> b) & 1u) << (3 * b + 2);
            kk |= (uint64_t)((qq[1] >> b) & 1u) << (3 * b + 1);
            kk |= (uint64_t)((qq[2] >> b) & 1u) << (3 * b);
        }
        key[i] = kk;
    }
}

/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; int64_t idx; } orc_pair;

static int orc_pair_cmp(const void *pa, const void *pb)
{
    const orc_pair *a = (const orc_pair *)pa, *b = (const orc_pair *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* perm[s] = original index of the s-th particle in (key, index) order. */
void orc_sort(int64_t n, const uint64_t *key, int64_t *perm)
{
    orc_pair *p = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { p[i].key = key[i]; p[i].idx = i; }
    qsort(p, (size_t)n, sizeof(orc_pair), orc_pair_cmp);
    for (int64_t i = 0; i < n; ++i) perm[i] = p[i].idx;
    free(p);
}

/* ------------------------------------------------------------------------ */
/* Octree, breadth-first numbering.
 *   node 0 = root: level 0, all n sorted particles.
 *   A node is internal iff count > lcap and level < 21; its children are its
 *   non-empty octants in octant order, octant = (key >> 3(20 - level)) & 7.
 *   Nodes are appended in the order they are created while the node array is
 *   scanned front to back, so level l precedes level l+1 and, within a level,
 *   prefixes ascend; the children of a node are contiguous.
 *   corner_d = q_d of any member with the low (21 - level) bits cleared.
 * skey: keys in sorted order.  Outputs are (cap)-sized arrays; the return value
 * is the node count, and nothing is written when it exceeds cap. */
typedef struct {
    int32_t *level; uint32_t *corner[3]; int64_t *first, *count, *child; int32_t *nchild;
    int64_t nn, cap;
} orc_tree;

static void orc_tree_grow(orc_tree *t)
{
    int64_t c = t->cap ? 2 * t->cap : 1024;
    t->level = (int32_t *)realloc(t->level, sizeof(int32_t) * c);
    for (int d = 0; d < 3; ++d) t->corner[d] = (uint32_t *)realloc(t->corner[d], sizeof(uint32_t) * c);
    t->first = (int64_t *)realloc(t->first, sizeof(int64_t) * c);
    t->count = (int64_t *)realloc(t->count, sizeof(int64_t) * c);
    t->child = (int64_t *)realloc(t->child, sizeof(int64_t) * c);
    t->nchild = (int32_t *)realloc(t->nchild, sizeof(int32_t) * c);
    t->cap = c;
}

static uint32_t orc_deinterleave(uint64_t key, int axis /* 0=x,1=y,2=z */)
{
    uint32_t v = 0;
    int off = 2 - axis;
    for (int b = 0; b < ORC_BITS; ++b) v |= (uint32_t)((key >> (3 * b + off)) & 1u) << b;
    return v;
}

static void orc_push(orc_tree *t, int32_t level, uint64_t key, int64_t first, int64_t count)
{
    if (t->nn == t->cap) orc_tree_grow(t);
    int64_t i = t->nn++;
    uint32_t mask = ~((1u << (ORC_BITS - level)) - 1u);
    t->level[i] = level;
    for (int d = 0; d < 3; ++d) t->corner[d][i] = orc_deinterleave(key, d) & mask;
    t->first[i] = first; t->count[i] = count; t->child[i] = -1; t->nchild[i] = 0;
}

int64_t orc_octree(int64_t n, const uint64_t *skey, int32_t lcap, int64_t cap,
                   int32_t *level, uint32_t *corner, int64_t *first, int64_t *count,
                   int64_t *child, int32_t *nchild)
{
    orc_tree t; memset(&t, 0, sizeof t);
    if (n > 0) orc_push(&t, 0, skey[0], 0, n);
    for (int64_t i = 0; i < t.nn; ++i) {
        int32_t lv = t.level[i];
        if (!(t.count[i] > lcap && lv < ORC_MAXLEVEL)) continue;
        int shift = 3 * (ORC_MAXLEVEL - 1 - lv);
        int64_t f = t.first[i], e = t.first[i] + t.count[i];
        int64_t c0 = t.nn;
        int64_t s = f;
        while (s < e) {
            unsigned oct = (unsigned)((skey[s] >> shift) & 7u);
            int64_t r = s;
            while (r < e && (unsigned)((skey[r] >> shift) & 7u) == oct) ++r;
            orc_push(&t, lv + 1, skey[s], s, r - s);
            s = r;
        }
        t.child[i] = c0;
        t.nchild[i] = (int32_t)(t.nn - c0);
    }
    int64_t nn = t.nn;
    if (nn <= cap) {
        for (int64_t i = 0; i < nn; ++i) {
            level[i] = t.level[i];
            for (int d = 0; d < 3; ++d) corner[d * cap + i] = t.corner[d][i];
            first[i] = t.first[i]; count[i] = t.count[i];
            child[i] = t.child[i]; nchild[i] = t.nchild[i];
        }
    }
    free(t.level); for (int d = 0; d < 3; ++d) free(t.corner[d]);
    free(t.first); free(t.count); free(t.child); free(t.nchild);
    return nn;
}

/* ------------------------------------------------------------------------ */
/* Cell moments straight from their definitions, over each cell's members:
 *   M = sum m_j,  R = sum m_j r_j / M,
 *   Q = sum m_j (3 y_j y_j^T - |y_j|^2 I),  y_j = r_j - R.
 * Q is stored as (xx, yy, zz, xy, xz, yz).  A massless cell gets R = its
 * geometric centre (passed in as centre) and Q = 0. */
void orc_moments(int64_t nn, const int64_t *first, const int64_t *count,
                 const double *centre /* (3, nn) */, const int64_t *perm,
                 int64_t n, const double *x, const double *m,
                 double *M, double *R /* (3, nn) */, double *Q /* (6, nn) */)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < nn; ++c) {
        double mt = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t s = first[c]; s < first[c] + count[c]; ++s) {
            int64_t j = perm[s];
            mt += m[j];
            sx += m[j] * x[j]; sy += m[j] * x[n + j]; sz += m[j] * x[2 * n + j];
        }
        double rx, ry, rz;
        if (mt != 0.0) { rx = sx / mt; ry = sy / mt; rz = sz / mt; }
        else { rx = centre[c]; ry = centre[nn + c]; rz = centre[2 * nn + c]; }
        double qxx = 0, qyy = 0, qzz = 0, qxy = 0, qxz = 0, qyz = 0;
        if (mt != 0.0) {
            for (int64_t s = first[c]; s < first[c] + count[c]; ++s) {
                int64_t j = perm[s];
                double yx = x[j] - rx, yy = x[n + j] - ry, yz = x[2 * n + j] - rz;
                double y2 = yx * yx + yy * yy + yz * yz;
                qxx += m[j] * (3.0 * yx * yx - y2);
                qyy += m[j] * (3.0 * yy * yy - y2);
                qzz += m[j] * (3.0 * yz * yz - y2);
                qxy += m[j] * (3.0 * yx * yy);
                qxz += m[j] * (3.0 * yx * yz);
                qyz += m[j] * (3.0 * yy * yz);
            }
        }
        M[c] = mt;
        R[c] = rx; R[nn + c] = ry; R[2 * nn + c] = rz;
        Q[c] = qxx; Q[nn + c] = qyy; Q[2 * nn + c] = qzz;
        Q[3 * nn + c] = qxy; Q[4 * nn + c] = qxz; Q[5 * nn + c] = qyz;
    }
}

/* ------------------------------------------------------------------------ */
/* Walk groups.  Particles are taken in key order in chunks of gs; a chunk is
 * further cut between consecutive particles i, i+1 that do not share the cell
 * delta levels above the finer of their two leaves, i.e. where
 *   P(i, i+1) < max(leaf_level(i), leaf_level(i+1)) - delta,
 * P = number of leading octal digits the two keys share (21 if equal), and
 * where the cell of level P holding both (their smallest common cell) has more
 * than cmax particles.  delta = 0 disables the first cut, cmax = 0 the second.
 * The population of that cell is the number of sorted keys whose first P
 * octal digits equal key i's: keys are sorted, so they form one run, whose
 * ends two binary searches over (key >> 3(21 - P)) find.
 * gfirst (capacity n + 1) receives the first sorted index of every group and n
 * at the end; returns the group count. */
static int64_t orc_prefix_bound(int64_t n, const uint64_t *skey, int sh, uint64_t pre, int upper)
{
    /* first j with (skey[j] >> sh) > pre (upper) or >= pre (lower) */
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        uint64_t v = sh >= 64 ? 0 : skey[mid] >> sh;
        int go_right = upper ? (v <= pre) : (v < pre);
        if (go_right) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

int64_t orc_groups(int64_t n, const uint64_t *skey, int64_t nn, const int32_t *level, const int64_t *first,
                   const int64_t *count, const int32_t *nchild, int32_t gs, int32_t delta, int64_t cmax,
                   int64_t *gfirst)
{
    int32_t *lv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    unsigned char *cut = (unsigned char *)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < nn; ++c)
        if (nchild[c] == 0)
            for (int64_t s = first[c]; s < first[c] + count[c]; ++s) lv[s] = level[c];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int start = (i % gs) == 0;
        if (!start && (delta > 0 || cmax > 0)) {
            uint64_t d = skey[i - 1] ^ skey[i];
            int common = 21;
            if (d) {
                int hb = 63 - __builtin_clzll(d);
                common = (62 - hb) / 3;
            }
            int lmax = lv[i - 1] > lv[i] ? lv[i - 1] : lv[i];
            if (delta > 0 && common < lmax - delta) start = 1;
            if (!start && cmax > 0) {
                const int sh = 3 * (21 - common);
                const uint64_t pre = sh >= 64 ? 0 : skey[i] >> sh;
                const int64_t cnt = orc_prefix_bound(n, skey, sh, pre, 1) - orc_prefix_bound(n, skey, sh, pre, 0);
                if (cnt > cmax) start = 1;
            }
        }
        cut[i] = (unsigned char)start;
    }
    int64_t ng = 0;
    for (int64_t i = 0; i < n; ++i)
        if (cut[i]) gfirst[ng++] = i;
    gfirst[ng] = n;
    free(cut);
    free(lv);
    return ng;
}

/* ------------------------------------------------------------------------ */
/* Group walk with the opening criterion.
 *   Group g = sorted particles [gfirst[g], gfirst[g+1]) (orc_groups); its
 *   integer box is [min q_d, max q_d + 1) per axis.  Node C at level l has side s = 2^(21-l)
 *   and box [c_d, c_d + s).  gap_d = max(0, c_d - ghi_d, glo_d - (c_d + s)),
 *   d2 = sum gap_d^2.  C is accepted as far iff s^2 < theta^2 d2 (FP64, with
 *   theta^2 = theta * theta rounded once); equality opens.  From the root:
 *   accepted -> PC list, rejected leaf -> PP list, rejected internal -> visit
 *   the children.  The walk is breadth first in node order, so both lists
 *   come out in ascending node index.
 * qs: (3, n) quantised coordinates in SORTED order.
 * gsel (nsel entries, or NULL for all ng groups in order): the groups to walk;
 * entry k of the CSR output belongs to group gsel[k].
 * Call once with pc_list = pp_list = NULL to get the offsets (CSR, nsel+1
 * entries each), then again with lists of the sizes pc_off[nsel], pp_off[nsel].
 * Each group's walk is independent of the others (OpenMP over groups).
 *
 * orc_walk_group: one group's walk; writes its lists at pc/pp when they are
 * non-NULL and returns the two list lengths.  queue: scratch of nn entries. */
static void orc_walk_group(const uint32_t *qs, int64_t n, int64_t s0, int64_t s1, double th2, int64_t nn,
                           const int32_t *level, const uint32_t *corner, const int64_t *child,
                           const int32_t *nchild, int64_t *queue, int64_t *pc, int64_t *pp,
                           int64_t *npc_out, int64_t *npp_out)
{
    int64_t glo[3], ghi[3];
    for (int d = 0; d < 3; ++d) {
        uint32_t mn = qs[d * n + s0], mx = qs[d * n + s0];
        for (int64_t s = s0; s < s1; ++s) {
            uint32_t v = qs[d * n + s];
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        glo[d] = mn; ghi[d] = (int64_t)mx + 1;
    }
    int64_t npc = 0, npp = 0, head = 0, tail = 0;
    if (nn > 0) queue[tail++] = 0;
    while (head < tail) {
        int64_t c = queue[head++];
        int64_t sd = (int64_t)1 << (ORC_BITS - level[c]);
        int64_t d2 = 0;
        for (int d = 0; d < 3; ++d) {
            int64_t cd = corner[d * nn + c];
            int64_t gap = 0;
            if (cd - ghi[d] > gap) gap = cd - ghi[d];
            if (glo[d] - (cd + sd) > gap) gap = glo[d] - (cd + sd);
            d2 += gap * gap;
        }
        int accept = (double)(sd * sd) < th2 * (double)d2;
        if (accept) {
            if (pc) pc[npc] = c;
            ++npc;
        } else if (nchild[c] == 0) {
            if (pp) pp[npp] = c;
            ++npp;
        } else {
            for (int32_t k = 0; k < nchild[c]; ++k) queue[tail++] = child[c] + k;
        }
    }
    *npc_out = npc; *npp_out = npp;
}

void orc_lists(int64_t n, const uint32_t *qs, int64_t ng, const int64_t *gfirst, int64_t nsel,
               const int64_t *gsel, double theta,
               int64_t nn, const int32_t *level, const uint32_t *corner /* (3, nn) */,
               const int64_t *child, const int32_t *nchild,
               int64_t *pc_off, int64_t *pp_off, int64_t *pc_list, int64_t *pp_list)
{
    const double th2 = theta * theta;
    if (!gsel) nsel = ng;
    /* the groups' walks are independent: lengths first, then offsets, then (second call) the lists */
#pragma omp parallel
    {
        int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn > 0 ? nn : 1));
#pragma omp for schedule(dynamic, 4)
        for (int64_t k = 0; k < nsel; ++k) {
            const int64_t g = gsel ? gsel[k] : k;
            int64_t a, b;
            orc_walk_group(qs, n, gfirst[g], gfirst[g + 1], th2, nn, level, corner, child, nchild, queue,
                           NULL, NULL, &a, &b);
            pc_off[k + 1] = a; pp_off[k + 1] = b;
        }
        free(queue);
    }
    pc_off[0] = 0; pp_off[0] = 0;
    for (int64_t k = 0; k < nsel; ++k) { pc_off[k + 1] += pc_off[k]; pp_off[k + 1] += pp_off[k]; }
    if (!pc_list || !pp_list) return;
#pragma omp parallel
    {
        int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn > 0 ? nn : 1));
#pragma omp for schedule(dynamic, 4)
        for (int64_t k = 0; k < nsel; ++k) {
            const int64_t g = gsel ? gsel[k] : k;
            int64_t a, b;
            orc_walk_group(qs, n, gfirst[g], gfirst[g + 1], th2, nn, level, corner, child, nchild, queue,
                           pc_list + pc_off[k], pp_list + pp_off[k], &a, &b);
        }
        free(queue);
    }
}

/* ------------------------------------------------------------------------ */
/* Cell expansion about the centre of mass R of cell C, y = r_i - R,
 * r_s^2 = |y|^2 + eps^2 (softened radius everywhere):
 *   a   = -G M y / r_s^3 + G (Q y) / r_s^5 - (5/2) G (y^T Q y) y / r_s^7
 *   phi = -G M / r_s - (1/2) G (y^T Q y) / r_s^5
 * (monopole: Q = 0).  PP part: Eq. 1 over the members of each near leaf,
 * j != i.  x, m in original order; outputs in original order.  gsel (nsel
 * entries, or NULL for all ng groups): the groups evaluated, with their lists
 * at CSR entry k as orc_lists gives them; other particles' outputs are left
 * as they are. */
void orc_tree_forces(int64_t n, const double *x, const double *m, const int64_t *perm,
                     int64_t ng, const int64_t *gfirst, int64_t nsel, const int64_t *gsel,
                     int64_t nn, const double *M, const double *R, const double *Q,
                     const int64_t *first, const int64_t *count,
                     const int64_t *pc_off, const int64_t *pc_list,
                     const int64_t *pp_off, const int64_t *pp_list,
                     double G, double eps, int32_t quad, double *a, double *phi)
{
    const double eps2 = eps * eps;
    if (!gsel) nsel = ng;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t kk = 0; kk < nsel; ++kk) {
        const int64_t g = gsel ? gsel[kk] : kk;
        int64_t s0 = gfirst[g], s1 = gfirst[g + 1];
        for (int64_t s = s0; s < s1; ++s) {
            int64_t i = perm[s];
            double xi = x[i], yi = x[n + i], zi = x[2 * n + i];
            double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0;
            for (int64_t e = pc_off[kk]; e < pc_off[kk + 1]; ++e) {
                int64_t c = pc_list[e];
                double yx = xi - R[c], yy = yi - R[nn + c], yz = zi - R[2 * nn + c];
                double r2 = yx * yx + yy * yy + yz * yz + eps2;
                double r = sqrt(r2);
                double i1 = 1.0 / r, i2 = 1.0 / r2;
                double i3 = i1 * i2, i5 = i3 * i2, i7 = i5 * i2;
                ax -= G * M[c] * yx * i3;
                ay -= G * M[c] * yy * i3;
                az -= G * M[c] * yz * i3;
                p -= G * M[c] * i1;
                if (quad) {
                    double qxx = Q[c], qyy = Q[nn + c], qzz = Q[2 * nn + c];
                    double qxy = Q[3 * nn + c], qxz = Q[4 * nn + c], qyz = Q[5 * nn + c];
                    double Qx = qxx * yx + qxy * yy + qxz * yz;
                    double Qy = qxy * yx + qyy * yy + qyz * yz;
                    double Qz = qxz * yx + qyz * yy + qzz * yz;
                    double yQy = yx * Qx + yy * Qy + yz * Qz;
                    ax += G * Qx * i5 - 2.5 * G * yQy * yx * i7;
                    ay += G * Qy * i5 - 2.5 * G * yQy * yy * i7;
                    az += G * Qz * i5 - 2.5 * G * yQy * yz * i7;
                    p -= 0.5 * G * yQy * i5;
                }
            }
            for (int64_t e = pp_off[kk]; e < pp_off[kk + 1]; ++e) {
                int64_t c = pp_list[e];
                for (int64_t t = first[c]; t < first[c] + count[c]; ++t) {
                    int64_t j = perm[t];
                    if (j == i) continue;
                    double dx = x[j] - xi, dy = x[n + j] - yi, dz = x[2 * n + j] - zi;
                    double r2 = dx * dx + dy * dy + dz * dz + eps2;
                    double r = sqrt(r2);
                    double w = G * m[j] / (r2 * r);
                    ax += w * dx; ay += w * dy; az += w * dz;
                    p -= G * m[j] / r;
                }
            }
            a[i] = ax; a[n + i] = ay; a[2 * n + i] = az;
            if (phi) phi[i] = p;
        }
    }
}

/* Number of OpenMP threads the parallel loops above use (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(void) { return omp_get_max_threads(); }
void orc_set_threads(int t) { if (t > 0) omp_set_num_threads(t); }
#else
int orc_threads(void) { return 1; }
void orc_set_threads(int t) { (void)t; }
#endif

/* ------------------------------------------------------------------------ */
/* Vector-Jacobian product of orc_tree_forces with the tree structure (order,
 * cells, groups, lists) held fixed and the moments recomputed from (x, m).
 * Given cotangents abar (3, n) of the accelerations and phibar (n) of the
 * potentials (caller order), adds to xbar (3, n) and mbar (n):
 *   PP pair (source j, target i, d = r_j - r_i, s^2 = |d|^2 + eps^2):
 *     g = G m_j (abar_i s^-3 - 3 d (d . abar_i) s^-5) + G m_j phibar_i d s^-3
 *     xbar_j += g, xbar_i -= g,
 *     mbar_j += G (d . abar_i) s^-3 - G phibar_i s^-1.
 *   PC pair (cell C, y = r_i - R): differentiate the cell expansion with
 *     respect to y (xbar_i += ybar, Rbar_C -= ybar), M (Mbar_C) and the six
 *     stored quadrupole components (Qbar_C).
 *   Cell cotangents reach the members j of C (y_j = r_j - R) through the
 *   definitions M = sum m_j, R = sum m_j r_j / M, Q = sum m_j (3 y_j y_j^T -
 *   |y_j|^2 I), with Qf the symmetric matrix of Qbar (off-diagonal entries
 *   halved) and f(y) = 3 y.Qf.y - |y|^2 tr(Qf):
 *     mbar_j += Mbar + y_j . Rbar / M + f(y_j)
 *     xbar_j += (m_j / M) Rbar + m_j (6 Qf y_j - 2 tr(Qf) y_j)
 *   (the dependence of Q on R drops out because sum m_j y_j = 0).
 *   Massless cells pass only Mbar on.  Serial (exact and simple). */
void orc_tree_forces_vjp(int64_t n, const double *x, const double *m, const int64_t *perm,
                         int64_t ng, const int64_t *gfirst, int64_t nn, const double *M, const double *R,
                         const double *Q, const int64_t *first, const int64_t *count,
                         const int64_t *pc_off, const int64_t *pc_list,
                         const int64_t *pp_off, const int64_t *pp_list,
                         double G, double eps, int32_t quad, const double *abar, const double *phibar,
                         double *xbar, double *mbar)
{
    const double eps2 = eps * eps;
    double *cb = (double *)calloc((size_t)(nn > 0 ? nn : 1) * 10, sizeof(double));  /* Mbar, Rbar[3], Qbar[6] */
    for (int64_t g = 0; g < ng; ++g) {
        for (int64_t s = gfirst[g]; s < gfirst[g + 1]; ++s) {
            const int64_t i = perm[s];
            const double xi = x[i], yi = x[n + i], zi = x[2 * n + i];
            const double bx = abar[i], by = abar[n + i], bz = abar[2 * n + i];
            const double pb = phibar ? phibar[i] : 0.0;
            for (int64_t e = pc_off[g]; e < pc_off[g + 1]; ++e) {
                const int64_t c = pc_list[e];
                const double yx = xi - R[c], yy = yi - R[nn + c], yz = zi - R[2 * nn + c];
                const double r2 = yx * yx + yy * yy + yz * yz + eps2;
                const double r = sqrt(r2);
                const double i1 = 1.0 / r, i2 = 1.0 / r2;
                const double i3 = i1 * i2, i5 = i3 * i2, i7 = i5 * i2, i9 = i7 * i2;
                const double Mc = M[c];
                const double yb = yx * bx + yy * by + yz * bz;
                /* monopole: a = -G M y i3, phi = -G M i1 */
                double gx = -G * Mc * (bx * i3 - 3.0 * yx * yb * i5) + G * Mc * pb * yx * i3;
                double gy = -G * Mc * (by * i3 - 3.0 * yy * yb * i5) + G * Mc * pb * yy * i3;
                double gz = -G * Mc * (bz * i3 - 3.0 * yz * yb * i5) + G * Mc * pb * yz * i3;
                double mb = -G * yb * i3 - G * pb * i1;
                double qb[6] = {0, 0, 0, 0, 0, 0};
                if (quad) {
                    const double qxx = Q[c], qyy = Q[nn + c], qzz = Q[2 * nn + c];
                    const double qxy = Q[3 * nn + c], qxz = Q[4 * nn + c], qyz = Q[5 * nn + c];
                    const double Qx = qxx * yx + qxy * yy + qxz * yz;
                    const double Qy = qxy * yx + qyy * yy + qyz * yz;
                    const double Qz = qxz * yx + qyz * yy + qzz * yz;
                    const double yQy = yx * Qx + yy * Qy + yz * Qz;
                    const double Qb = Qx * bx + Qy * by + Qz * bz;      /* (Q y) . abar */
                    /* a_q = G Q y i5 - 2.5 G yQy y i7 ;  phi_q = -0.5 G yQy i5
                     * d/dy of abar.a_q = G [Q abar i5 - 5 (Qy.abar) y i7 - 2.5 (2 Qy (y.abar) + yQy abar) i7
                     *                       + 17.5 yQy (y.abar) y i9]
                     * d/dy of pb phi_q = pb G [-Qy i5 + 2.5 yQy y i7] */
                    const double Qbx = qxx * bx + qxy * by + qxz * bz;
                    const double Qby = qxy * bx + qyy * by + qyz * bz;
                    const double Qbz = qxz * bx + qyz * by + qzz * bz;
                    gx += G * (Qbx * i5 - 5.0 * Qb * yx * i7 - 2.5 * (2.0 * Qx * yb + yQy * bx) * i7 + 17.5 * yQy * yb * yx * i9)
                        + pb * G * (-Qx * i5 + 2.5 * yQy * yx * i7);
                    gy += G * (Qby * i5 - 5.0 * Qb * yy * i7 - 2.5 * (2.0 * Qy * yb + yQy * by) * i7 + 17.5 * yQy * yb * yy * i9)
                        + pb * G * (-Qy * i5 + 2.5 * yQy * yy * i7);
                    gz += G * (Qbz * i5 - 5.0 * Qb * yz * i7 - 2.5 * (2.0 * Qz * yb + yQy * bz) * i7 + 17.5 * yQy * yb * yz * i9)
                        + pb * G * (-Qz * i5 + 2.5 * yQy * yz * i7);
                    /* d/dQ (stored components): abar.a_q = G i5 (y^T Qf abar) - 2.5 G i7 yb (y^T Qf y)
                     * and pb phi_q = -0.5 G pb i5 (y^T Qf y); a diagonal entry appears once,
                     * an off-diagonal stored entry twice (Q[a][b] and Q[b][a]). */
                    const double ca = G * i5, cb2 = -2.5 * G * i7 * yb - 0.5 * G * pb * i5;
                    qb[0] = ca * yx * bx + cb2 * yx * yx;
                    qb[1] = ca * yy * by + cb2 * yy * yy;
                    qb[2] = ca * yz * bz + cb2 * yz * yz;
                    qb[3] = ca * (yx * by + yy * bx) + cb2 * 2.0 * yx * yy;
                    qb[4] = ca * (yx * bz + yz * bx) + cb2 * 2.0 * yx * yz;
                    qb[5] = ca * (yy * bz + yz * by) + cb2 * 2.0 * yy * yz;
                }
                xbar[i] += gx; xbar[n + i] += gy; xbar[2 * n + i] += gz;
                double *cc = cb + 10 * c;
                cc[0] += mb;
                cc[1] -= gx; cc[2] -= gy; cc[3] -= gz;
                for (int k = 0; k < 6; ++k) cc[4 + k] += qb[k];
            }
            for (int64_t e = pp_off[g]; e < pp_off[g + 1]; ++e) {
                const int64_t c = pp_list[e];
                for (int64_t t = first[c]; t < first[c] + count[c]; ++t) {
                    const int64_t j = perm[t];
                    if (j == i) continue;
                    const double dx = x[j] - xi, dy = x[n + j] - yi, dz = x[2 * n + j] - zi;
                    const double r2 = dx * dx + dy * dy + dz * dz + eps2;
                    const double r = sqrt(r2);
                    const double i1 = 1.0 / r, i3 = i1 / r2, i5 = i3 / r2;
                    const double db = dx * bx + dy * by + dz * bz;
                    const double gm = G * m[j];
                    const double gx = gm * (bx * i3 - 3.0 * dx * db * i5) + gm * pb * dx * i3;
                    const double gy = gm * (by * i3 - 3.0 * dy * db * i5) + gm * pb * dy * i3;
                    const double gz = gm * (bz * i3 - 3.0 * dz * db * i5) + gm * pb * dz * i3;
                    xbar[j] += gx; xbar[n + j] += gy; xbar[2 * n + j] += gz;
                    xbar[i] -= gx; xbar[n + i] -= gy; xbar[2 * n + i] -= gz;
                    mbar[j] += G * db * i3 - G * pb * i1;
                }
            }
        }
    }
    /* push every cell's cotangent to its members, from the definitions */
    for (int64_t c = 0; c < nn; ++c) {
        const double *cc = cb + 10 * c;
        int nz = 0;
        for (int k = 0; k < 10; ++k) nz |= cc[k] != 0.0;
        if (!nz) continue;
        const double Mc = M[c];
        for (int64_t t = first[c]; t < first[c] + count[c]; ++t) {
            const int64_t j = perm[t];
            mbar[j] += cc[0];
            if (Mc == 0.0) continue;
            const double yx = x[j] - R[c], yy = x[n + j] - R[nn + c], yz = x[2 * n + j] - R[2 * nn + c];
            /* symmetric cotangent matrix: diagonal as stored, off-diagonal halved */
            const double fxx = cc[4], fyy = cc[5], fzz = cc[6];
            const double fxy = 0.5 * cc[7], fxz = 0.5 * cc[8], fyz = 0.5 * cc[9];
            const double tr = fxx + fyy + fzz;
            const double Fx = fxx * yx + fxy * yy + fxz * yz;
            const double Fy = fxy * yx + fyy * yy + fyz * yz;
            const double Fz = fxz * yx + fyz * yy + fzz * yz;
            const double y2 = yx * yx + yy * yy + yz * yz;
            const double f = 3.0 * (yx * Fx + yy * Fy + yz * Fz) - y2 * tr;
            mbar[j] += (yx * cc[1] + yy * cc[2] + yz * cc[3]) / Mc + f;
            const double w = m[j] / Mc;
            xbar[j] += w * cc[1] + m[j] * (6.0 * Fx - 2.0 * tr * yx);
            xbar[n + j] += w * cc[2] + m[j] * (6.0 * Fy - 2.0 * tr * yy);
            xbar[2 * n + j] += w * cc[3] + m[j] * (6.0 * Fz - 2.0 * tr * yz);
        }
    }
    free(cb);
}
