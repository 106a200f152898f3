// circuits.cu -- boolean circuits over encrypted integers, compiled into a
// level schedule of batched bootstraps.
//
// Circuits (bit 0 least significant, all results mod 2^w):
//  * add: ripple-carry adder, r_i = a_i ^ b_i ^ c_(i-1) (Eq. "addres"),
//    c_i = a_i b_i | (a_i ^ b_i) c_(i-1) (Eq. "addcarry"); no carry in, no
//    carry out (sections III-A and V-B-1);
//  * mul: naive multiplication (section III-B-1): partial product i = A AND
//    b_i shifted left by i, truncated to w bits and accumulated one after
//    another with ripple-carry adders;
//  * matvec: y_r = sum_c M[r][c] v[c] (section IV-D) with the products of a
//    row reduced by tree-based accumulation (section V-B-2): neighbours
//    (0,1), (2,3), ... are added per level, an odd last term moves up.
// Variants, each defined gate by gate below: the majority-carry adder (a
// carry is one 3-input MAJ bootstrap), the number-wise adder GPU_n
// (section V-B-1), tree-accumulated multiplication (section V-B-2) with
// ripple or majority-carry adders, full w x w -> 2w products (naive and
// Karatsuba, section III-B-2), and the low-depth parallel-prefix adder and
// Dadda-tree multiplier.
//
// GB300 design: gates of one level from all instances and all jobs of a
// batch form one blind-rotation launch and one key-switch launch that
// gather their inputs from, and scatter their outputs to, a
// device-resident ciphertext pool.  Levels are ASAP (1 + the deeper
// input) or, by default, deadline-driven: every gate keeps its ASAP depth
// bound and levels are filled to whole waves of the GPU (a level unit of
// 152, 608 or 760 gates, chosen per job mix from the autotuner's measured
// level and wave times).  The compiled schedule is cached per job
// signature and its level sequence is captured once as a CUDA graph and
// replayed.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "netlist.h"
#include "runtime.h"

namespace tgb {

// ---------------------------------------------------------------------
// Netlists
// ---------------------------------------------------------------------

// Ripple-carry adder on wire vectors x, y (w bits); returns sum wires.
static std::vector<int> build_add(Netlist &nl, const std::vector<int> &x, const std::vector<int> &y)
{
    const int w = (int)x.size();
    std::vector<int> r(w);
    int c = -1;
    for (int i = 0; i < w; ++i) {
        if (i == 0) {
            r[0] = nl.gate(TFHE_XOR, x[0], y[0]);
            if (w > 1)
                c = nl.gate(TFHE_AND, x[0], y[0]);
            continue;
        }
        const int p = nl.gate(TFHE_XOR, x[i], y[i]);   // propagate a_i ^ b_i
        r[i] = nl.gate(TFHE_XOR, p, c);                // sum bit
        if (i == w - 1)
            break;                                     // carry out is dropped
        const int g = nl.gate(TFHE_AND, x[i], y[i]);   // generate a_i b_i
        const int t = nl.gate(TFHE_AND, p, c);
        c = nl.gate(TFHE_OR, g, t);
    }
    return r;
}

// Truncated shift-and-add multiplier: w x w -> w bits.
static std::vector<int> build_mul(Netlist &nl, const std::vector<int> &x, const std::vector<int> &y)
{
    const int w = (int)x.size();
    std::vector<int> acc(w);
    for (int j = 0; j < w; ++j)
        acc[j] = nl.gate(TFHE_AND, x[j], y[0]);
    for (int i = 1; i < w; ++i) {
        const int m = w - i;
        std::vector<int> pp(m), hi(acc.begin() + i, acc.end());
        for (int j = 0; j < m; ++j)
            pp[j] = nl.gate(TFHE_AND, x[j], y[i]);     // a_j b_i has weight i + j
        std::vector<int> s = build_add(nl, hi, pp);
        std::copy(s.begin(), s.end(), acc.begin() + i);
    }
    return acc;
}

// One adder cell over operands that may be the constant 0 (wire -1): with
// one live operand the sum is that wire, with two a half adder (XOR, AND),
// with three a full adder, either the ripple form of Eq. "addres" /
// "addcarry" (p = x^y, s = p^c, carry = (x&y) | (p&c)) or the majority form
// (carry = MAJ(x, y, c), one bootstrap).  The carry is built only if needed.
static void adder_cell(Netlist &nl, int x, int y, int cin, bool need_carry, bool maj, int &s,
                       int &cout)
{
    int live[3], k = 0;
    for (int w : {x, y, cin})
        if (w >= 0)
            live[k++] = w;
    s = cout = -1;
    if (k == 1) {
        s = live[0];
    } else if (k == 2) {
        s = nl.gate(TFHE_XOR, live[0], live[1]);
        if (need_carry)
            cout = nl.gate(TFHE_AND, live[0], live[1]);
    } else if (k == 3) {
        const int p = nl.gate(TFHE_XOR, x, y);
        s = nl.gate(TFHE_XOR, p, cin);
        if (need_carry) {
            if (maj) {
                cout = nl.gate(TFHE_MAJ, x, y, cin);
            } else {
                const int g = nl.gate(TFHE_AND, x, y);
                const int t = nl.gate(TFHE_AND, p, cin);
                cout = nl.gate(TFHE_OR, g, t);
            }
        }
    }
}

// w-bit sum (mod 2^w) of two wire vectors with constant-zero entries.
static std::vector<int> build_add_const(Netlist &nl, const std::vector<int> &x,
                                        const std::vector<int> &y, bool maj)
{
    const int w = (int)x.size();
    std::vector<int> r(w);
    int c = -1;
    for (int i = 0; i < w; ++i)
        adder_cell(nl, x[i], y[i], c, i < w - 1, maj, r[i], c);
    return r;
}

// The paper's number-wise addition GPU_n (section V-B-1): R = A, then w
// times: C = R AND B, R = R XOR B, B = C << 1 -- both gates on all live
// bits at once (a compound gate).  Bits of B known to be 0 (shifted in)
// generate no gates; the carry out of bit w-1 is dropped.
static std::vector<int> build_add_numberwise(Netlist &nl, const std::vector<int> &x,
                                             const std::vector<int> &y)
{
    const int w = (int)x.size();
    std::vector<int> R(x), B(y);
    for (int k = 0; k < w; ++k) {
        std::vector<int> nR(R), nB(w, -1);
        for (int i = 0; i < w; ++i) {
            if (B[i] < 0)
                continue;
            nR[i] = nl.gate(TFHE_XOR, R[i], B[i]);
            if (i + 1 < w)
                nB[i + 1] = nl.gate(TFHE_AND, R[i], B[i]);
        }
        R.swap(nR);
        B.swap(nB);
    }
    return R;
}

// Truncated multiplication with tree-based accumulation (section V-B-2):
// partial products A AND b_i shifted by i (low i bits constant 0) are
// summed pairwise, (0,1), (2,3), ..., an odd last term moving up, with
// ripple-carry adders that skip constant-zero bits (carries of Eq.
// "addcarry", or single majority gates when maj).
static std::vector<int> build_mul_tree(Netlist &nl, const std::vector<int> &x,
                                       const std::vector<int> &y, bool maj)
{
    const int w = (int)x.size();
    std::vector<std::vector<int>> terms;
    for (int i = 0; i < w; ++i) {
        std::vector<int> pp(w, -1);
        for (int j = 0; i + j < w; ++j)
            pp[i + j] = nl.gate(TFHE_AND, x[j], y[i]);
        terms.push_back(pp);
    }
    while (terms.size() > 1) {
        std::vector<std::vector<int>> next;
        for (size_t i = 0; i + 1 < terms.size(); i += 2)
            next.push_back(build_add_const(nl, terms[i], terms[i + 1], maj));
        if (terms.size() & 1)
            next.push_back(terms.back());
        terms.swap(next);
    }
    return terms[0];
}

// Parallel-prefix adder (Sklansky): the w-bit sum mod 2^w of wire vectors
// with constant-zero entries (-1), on majority gates only.  Bit i gives
// generate g_i = x_i AND y_i (i < w - 1: there is no carry out),
// carry-or-transmit k_i = x_i OR y_i (0 < i < w - 1: a group that starts
// at bit 0 never needs its K) and p_i = x_i XOR y_i for its sum.  A group of bits has generate G (it makes a carry) and K = G OR
// (every bit transmits), so G implies K and the merge of a high group with
// the low group below it is two majority gates:
//   G = G_hi OR (K_hi AND G_lo) = MAJ(G_hi, K_hi, G_lo),
//   K = G_hi OR (K_hi AND K_lo) = MAJ(G_hi, K_hi, K_lo).
// Prefix level k (while 2^k < w - 1) merges, for every bit i <= w - 2 with
// bit k set, the group ending at i with the one ending at
// j = (i with its low k + 1 bits cleared) + 2^k - 1; K is formed only where
// the merged group does not start at bit 0.  The sum is
// s_i = p_i XOR G_(i-1) (s_0 = p_0).  Constant zeros are folded (a merge
// with G_lo = 0 keeps G_hi; with G_hi = 0 it is K_hi AND G_lo), so no gate
// gets a constant input.  Every gate keeps the 1/8 margin of the majority
// and two-input gates.
static std::vector<int> build_add_prefix(Netlist &nl, const std::vector<int> &x,
                                         const std::vector<int> &y)
{
    const int w = (int)x.size();
    std::vector<int> G(w, -1), K(w, -1), p(w, -1);
    for (int i = 0; i < w; ++i) {
        if (x[i] >= 0 && y[i] >= 0) {
            if (i + 1 < w)
                G[i] = nl.gate(TFHE_AND, x[i], y[i]);
            if (i > 0 && i + 1 < w)
                K[i] = nl.gate(TFHE_OR, x[i], y[i]);
            p[i] = nl.gate(TFHE_XOR, x[i], y[i]);
        } else {
            p[i] = x[i] >= 0 ? x[i] : y[i];
            if (i + 1 < w)
                K[i] = p[i];
        }
    }
    // G_hi OR (K_hi AND L), folding constant zeros
    auto merge = [&nl](int g_hi, int k_hi, int lo) {
        if (lo < 0 || k_hi < 0)
            return g_hi;
        if (g_hi < 0)
            return nl.gate(TFHE_AND, k_hi, lo);
        return nl.gate(TFHE_MAJ, g_hi, k_hi, lo);
    };
    for (int k = 0; (1 << k) < w - 1; ++k) {
        std::vector<int> nG(G), nK(K);
        for (int i = 0; i <= w - 2; ++i) {
            if (!((i >> k) & 1))
                continue;
            const int j = ((i >> (k + 1)) << (k + 1)) + (1 << k) - 1;
            nG[i] = merge(G[i], K[i], G[j]);
            if ((i >> (k + 1)) != 0)
                nK[i] = merge(G[i], K[i], K[j]);
        }
        G.swap(nG);
        K.swap(nK);
    }
    std::vector<int> s(w);
    for (int i = 0; i < w; ++i) {
        const int c = i ? G[i - 1] : -1;
        s[i] = c < 0 ? p[i] : p[i] < 0 ? c : nl.gate(TFHE_XOR, p[i], c);
    }
    return s;
}

// Truncated multiplication (w x w -> w bits) by a Dadda tree.  Column c
// starts with the partial products a_(c-i) AND b_i, i = 0 .. c.  Stage
// targets are the terms of d_1 = 2, d_(k+1) = floor(3 d_k / 2) below w,
// largest first.  In a stage every column, in increasing order, is reduced
// to at most d wires, its height counting the carries the previous column
// sent it in this stage: a half adder (sum x XOR y, carry x AND y) when one
// wire too many, else a full adder (sum (x XOR y) XOR z, carry MAJ(x, y, z)),
// on the column's oldest wires.  The new column lists the carries received,
// then its sums, then its untouched wires.  Carries out of column w - 1 are
// not built.  The two rows left go to the parallel-prefix adder.  Returns
// false if a column lacks wires for its adders (no width up to 64 does).
static bool build_mul_dadda(Netlist &nl, const std::vector<int> &x, const std::vector<int> &y,
                            std::vector<int> &out)
{
    const int w = (int)x.size();
    std::vector<std::vector<int>> col(w);
    for (int c = 0; c < w; ++c)
        for (int i = 0; i <= c; ++i)
            col[c].push_back(nl.gate(TFHE_AND, x[c - i], y[i]));
    std::vector<int> targets;
    for (int d = 2; d < w; d = d * 3 / 2)
        targets.push_back(d);
    for (auto t = targets.rbegin(); t != targets.rend(); ++t) {
        const int d = *t;
        std::vector<std::vector<int>> nc(w);
        for (int c = 0; c < w; ++c) {
            const std::vector<int> &L = col[c];
            size_t pos = 0;
            int h = (int)(L.size() + nc[c].size());
            while (h > d) {
                const bool half = h - d == 1;
                if (pos + (half ? 2 : 3) > L.size())
                    return false;
                const int u = L[pos], v = L[pos + 1];
                if (half) {
                    nc[c].push_back(nl.gate(TFHE_XOR, u, v));
                    if (c + 1 < w)
                        nc[c + 1].push_back(nl.gate(TFHE_AND, u, v));
                    pos += 2;
                    h -= 1;
                } else {
                    const int z = L[pos + 2];
                    nc[c].push_back(nl.gate(TFHE_XOR, nl.gate(TFHE_XOR, u, v), z));
                    if (c + 1 < w)
                        nc[c + 1].push_back(nl.gate(TFHE_MAJ, u, v, z));
                    pos += 3;
                    h -= 2;
                }
            }
            for (; pos < L.size(); ++pos)
                nc[c].push_back(L[pos]);
        }
        col.swap(nc);
    }
    std::vector<int> r0(w, -1), r1(w, -1);
    for (int c = 0; c < w; ++c) {
        if (col[c].size() > 2)
            return false;
        if (col[c].size() > 0)
            r0[c] = col[c][0];
        if (col[c].size() > 1)
            r1[c] = col[c][1];
    }
    out = build_add_prefix(nl, r0, r1);
    return true;
}

// Full product of two wire vectors (len(x) = len(y) = n -> 2n bits):
// partial products at their weights, summed by the same pairwise tree.
static std::vector<int> build_mul_full(Netlist &nl, const std::vector<int> &x,
                                       const std::vector<int> &y)
{
    const int n = (int)x.size(), w = 2 * n;
    std::vector<std::vector<int>> terms;
    for (int i = 0; i < n; ++i) {
        std::vector<int> pp(w, -1);
        for (int j = 0; j < n; ++j)
            pp[i + j] = nl.gate(TFHE_AND, x[j], y[i]);
        terms.push_back(pp);
    }
    while (terms.size() > 1) {
        std::vector<std::vector<int>> next;
        for (size_t i = 0; i + 1 < terms.size(); i += 2)
            next.push_back(build_add_const(nl, terms[i], terms[i + 1], false));
        if (terms.size() & 1)
            next.push_back(terms.back());
        terms.swap(next);
    }
    return terms[0];
}

// Sum with carry out: max(len) + 1 bits.
static std::vector<int> build_add_ext(Netlist &nl, std::vector<int> x, std::vector<int> y)
{
    const size_t L = std::max(x.size(), y.size()) + 1;
    x.resize(L, -1);
    y.resize(L, -1);
    return build_add_const(nl, x, y, false);
}

// a - b mod 2^len(a) = a + NOT b + 1 for len(b) <= len(a), every bit of a
// live.  Cells: with the carry-in 1 of bit 0, sum a XOR b and carry
// a OR NOT b (ORYN); with a live carry, p = a XNOR b, sum p XOR c, carry
// (a AND NOT b) OR (p AND c); past the end of b (NOT 0 = 1), sum a XNOR c
// and carry a OR c.  Returns false if a case outside these arises.
static bool build_sub(Netlist &nl, const std::vector<int> &a, const std::vector<int> &b,
                      std::vector<int> &r)
{
    const int L = (int)a.size();
    r.assign(L, -1);
    int c = -2;  // -2: the constant 1
    for (int i = 0; i < L; ++i) {
        const bool need = i < L - 1;
        const int bi = i < (int)b.size() ? b[i] : -1;
        if (a[i] < 0)
            return false;
        if (bi >= 0 && c == -2) {
            r[i] = nl.gate(TFHE_XOR, a[i], bi);
            c = need ? nl.gate(TFHE_ORYN, a[i], bi) : -1;
        } else if (bi >= 0 && c >= 0) {
            const int p = nl.gate(TFHE_XNOR, a[i], bi);
            r[i] = nl.gate(TFHE_XOR, p, c);
            if (need) {
                const int g = nl.gate(TFHE_ANDYN, a[i], bi);
                const int t = nl.gate(TFHE_AND, p, c);
                c = nl.gate(TFHE_OR, g, t);
            }
        } else if (bi < 0 && c >= 0) {
            r[i] = nl.gate(TFHE_XNOR, a[i], c);
            c = need ? nl.gate(TFHE_OR, a[i], c) : -1;
        } else {
            return false;
        }
    }
    return true;
}

// Karatsuba multiplication (Algorithm "karatsuba"; the printed recombination
// is garbled -- here the textbook form): for n-bit X, Y with n >= n0,
// h = ceil(n/2), X = X0 + X1 2^h, Y likewise;
//   Z0 = K(X0, Y0), Z1 = K(X1, Y1), Z2 = K(X0 + X1, Y0 + Y1)  (sums carry out)
//   M  = Z2 - (Z0 + Z1) = X0 Y1 + X1 Y0
//   Z  = (Z0 + Z1 2^(2h)) + M 2^h                 (2n bits)
// The first term is Z0 and Z1 side by side (no gates).  Below n0 the full
// product is formed directly.
static bool build_karatsuba(Netlist &nl, const std::vector<int> &x, const std::vector<int> &y,
                            int n0, std::vector<int> &z)
{
    const int n = (int)x.size();
    if (n < n0) {
        z = build_mul_full(nl, x, y);
        return true;
    }
    const int h = (n + 1) / 2;
    std::vector<int> x0(x.begin(), x.begin() + h), x1(x.begin() + h, x.end());
    std::vector<int> y0(y.begin(), y.begin() + h), y1(y.begin() + h, y.end());
    std::vector<int> z0, z1, z2, m;
    if (!build_karatsuba(nl, x0, y0, n0, z0) || !build_karatsuba(nl, x1, y1, n0, z1))
        return false;
    std::vector<int> sx = build_add_ext(nl, x0, x1), sy = build_add_ext(nl, y0, y1);
    if (!build_karatsuba(nl, sx, sy, n0, z2))
        return false;
    std::vector<int> u = build_add_ext(nl, z0, z1);
    if (!build_sub(nl, z2, u, m))
        return false;
    std::vector<int> t(z0);
    t.insert(t.end(), z1.begin(), z1.end());       // Z0 + Z1 2^(2h), 2n bits
    std::vector<int> ms(2 * n, -1);
    for (int i = 0; i < (int)m.size() && h + i < 2 * n; ++i)
        ms[h + i] = m[i];
    z = build_add_const(nl, t, ms, false);
    return true;
}

static std::vector<int> range_wires(int start, int count)
{
    std::vector<int> v(count);
    for (int k = 0; k < count; ++k)
        v[k] = start + k;
    return v;
}

// Input wires: ADD/MUL: A bits [0, w), B bits [w, 2w).  GATE: a = 0, b = 1.
// MATVEC: M[r][c] bits at (r*cols + c)*w + bit, then v[c] bits.
bool build_netlist(int kind, int w, int rows, int cols, Netlist &nl)
{
    switch (kind) {
    case TFHE_CIRCUIT_GATE:   // any two-input opcode (not the 3-input MAJ)
        if (w < 0 || w > TFHE_ORYN || w == TFHE_MAJ)
            return false;
        nl.n_in = 2;
        nl.out = {nl.gate(w, 0, 1)};
        break;
    case TFHE_CIRCUIT_ADD:
    case TFHE_CIRCUIT_MUL:
        if (w < 1 || w > 64)
            return false;
        nl.n_in = 2 * w;
        nl.out = kind == TFHE_CIRCUIT_ADD ? build_add(nl, range_wires(0, w), range_wires(w, w))
                                          : build_mul(nl, range_wires(0, w), range_wires(w, w));
        break;
    case TFHE_CIRCUIT_ADD_MAJ:
    case TFHE_CIRCUIT_ADD_NW:
    case TFHE_CIRCUIT_MUL_TREE:
    case TFHE_CIRCUIT_MUL_TREE_MAJ:
        if (w < 1 || w > 64)
            return false;
        nl.n_in = 2 * w;
        nl.out = kind == TFHE_CIRCUIT_ADD_MAJ
                     ? build_add_const(nl, range_wires(0, w), range_wires(w, w), true)
                 : kind == TFHE_CIRCUIT_ADD_NW
                     ? build_add_numberwise(nl, range_wires(0, w), range_wires(w, w))
                     : build_mul_tree(nl, range_wires(0, w), range_wires(w, w),
                                      kind == TFHE_CIRCUIT_MUL_TREE_MAJ);
        for (int o : nl.out)
            if (o < 0)
                return false;
        break;
    case TFHE_CIRCUIT_ADD_PREFIX:
    case TFHE_CIRCUIT_MUL_DADDA:
        if (w < 1 || w > 64)
            return false;
        nl.n_in = 2 * w;
        if (kind == TFHE_CIRCUIT_ADD_PREFIX)
            nl.out = build_add_prefix(nl, range_wires(0, w), range_wires(w, w));
        else if (!build_mul_dadda(nl, range_wires(0, w), range_wires(w, w), nl.out))
            return false;
        for (int o : nl.out)
            if (o < 0)
                return false;
        break;
    case TFHE_CIRCUIT_MUL_FULL:
    case TFHE_CIRCUIT_MUL_KARATSUBA: {
        if (w < 2 || w > 64)   // at w = 1 the top product bit is the constant 0
            return false;
        nl.n_in = 2 * w;
        if (kind == TFHE_CIRCUIT_MUL_FULL)
            nl.out = build_mul_full(nl, range_wires(0, w), range_wires(w, w));
        else if (!build_karatsuba(nl, range_wires(0, w), range_wires(w, w), 8, nl.out))
            return false;
        for (int o : nl.out)
            if (o < 0)
                return false;
        break;
    }
    case TFHE_CIRCUIT_MATVEC: {
        if (w < 1 || w > 64 || rows < 1 || cols < 1 || (long)rows * cols > 4096)
            return false;
        nl.n_in = (rows * cols + cols) * w;
        const int vbase = rows * cols * w;
        for (int r = 0; r < rows; ++r) {
            std::vector<std::vector<int>> terms;
            for (int c = 0; c < cols; ++c)
                terms.push_back(build_mul(nl, range_wires((r * cols + c) * w, w),
                                          range_wires(vbase + c * w, w)));
            while (terms.size() > 1) {
                std::vector<std::vector<int>> next;
                for (size_t i = 0; i + 1 < terms.size(); i += 2)
                    next.push_back(build_add(nl, terms[i], terms[i + 1]));
                if (terms.size() & 1)
                    next.push_back(terms.back());
                terms.swap(next);
            }
            nl.out.insert(nl.out.end(), terms[0].begin(), terms[0].end());
        }
        break;
    }
    default:
        return false;
    }
    nl.levelise();
    return true;
}

// Rows per instance of the two input groups.
void input_groups(int kind, int w, int rows, int cols, long &rows0, long &rows1)
{
    if (kind == TFHE_CIRCUIT_MATVEC) {
        rows0 = (long)rows * cols * w;
        rows1 = (long)cols * w;
    } else {
        rows0 = rows1 = kind == TFHE_CIRCUIT_GATE ? 1 : w;
    }
}

// ---------------------------------------------------------------------
// Compiled plans
// ---------------------------------------------------------------------

__global__ void k_gather_rows_impl(int32_t *dst, const int32_t *__restrict__ src, long src_rows,
                                   const int32_t *__restrict__ rows, long count,
                                   uint32_t *status)
{
    const long r = blockIdx.x;
    if (r >= count)
        return;
    const long sr = rows[r];
    if (sr < 0 || sr >= src_rows) {
        if (threadIdx.x == 0)
            atomicOr(status, kErrGather);
        return;
    }
    const int4 *s = reinterpret_cast<const int4 *>(src + sr * kLweStride);
    int4 *d = reinterpret_cast<int4 *>(dst + r * kLweStride);
    for (int k = threadIdx.x; k < kLweStride / 4; k += blockDim.x)
        d[k] = s[k];
}

cudaError_t launch_gather_rows(int32_t *dst, const int32_t *src, long src_rows,
                               const int32_t *rows, long count, uint32_t *status,
                               cudaStream_t st)
{
    if (count <= 0)
        return cudaSuccess;
    k_gather_rows_impl<<<(unsigned)count, 128, 0, st>>>(dst, src, src_rows, rows, count, status);
    return cudaGetLastError();
}

std::shared_ptr<const Netlist> get_netlist(int kind, int w, int rows, int cols)
{
    static std::mutex mu;
    static std::map<std::string, std::shared_ptr<const Netlist>> cache;
    char key[64];
    std::snprintf(key, sizeof(key), "%d:%d:%d:%d", kind, w, rows, cols);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end())
        return it->second;
    auto nl = std::make_shared<Netlist>();
    if (!build_netlist(kind, w, rows, cols, *nl))
        return nullptr;
    cache.emplace(key, nl);
    return nl;
}

struct JobLayout {
    int kind, w, rows, cols;
    long batch;
    long base;           // first pool row of instance 0
    long inst_rows;      // pool rows per instance
    long rows0, rows1;   // input rows per instance (group 0, group 1)
    long n_out;          // outputs per instance
    long out_off;        // offset of this job's output rows in d_out_rows
};

struct Plan {
    std::vector<JobLayout> jobs;
    long pool_rows = 0, gates = 0, max_width = 0;
    int depth = 0;
    std::vector<long> level_off;     // depth + 1 entries
    int32_t *pool = nullptr;
    int32_t *big = nullptr;
    uint8_t *d_ops = nullptr;
    int32_t *d_ia = nullptr, *d_ib = nullptr, *d_ic = nullptr, *d_io = nullptr,
            *d_out_rows = nullptr;
    std::vector<uint8_t> h_ops;      // host copies for the per-gate schedule
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    bool graph_profiled = false;     // graph carries event-record nodes
    long kernels_per_run = 0;        // kernel launches of one level sequence
    long wave = 0;                   // gates per level unit the schedule rounds to
    int wide_shape = 0;              // blind-rotation shape of levels of >= wave gates
    std::vector<cudaEvent_t> ev;     // 3 per level: BR start, BR end / KS start, KS end

    ~Plan()
    {
        if (graph)
            cudaGraphExecDestroy(graph);
        for (cudaEvent_t e : ev)
            cudaEventDestroy(e);
        cudaFree(pool);
        cudaFree(big);
        cudaFree(d_ops);
        cudaFree(d_ia);
        cudaFree(d_ib);
        cudaFree(d_ic);
        cudaFree(d_io);
        cudaFree(d_out_rows);
    }
};

struct CircuitCache {
    std::map<std::string, std::unique_ptr<Plan>> plans;
    std::vector<std::string> order;  // insertion order for eviction
    bool use_graphs = true;
    bool per_gate = false;
    bool profile = false;
    int policy = TFHE_SCHED_BALANCED;
    long level_width = 0;            // 0: one wave, of 4 or 5 bootstraps per SM
    std::map<std::string, long> wave_choice;   // job signature -> chosen wave
    std::vector<Plan *> profiled;    // plans whose events hold the last run
    cudaStream_t capture_stream = nullptr;
    ~CircuitCache()
    {
        plans.clear();
        if (capture_stream)
            cudaStreamDestroy(capture_stream);
    }
};

static CircuitCache &cache_of(tfhe_ctx *ctx)
{
    if (!ctx->circuits)
        ctx->circuits = new CircuitCache();
    return *ctx->circuits;
}

void invalidate_graphs(tfhe_ctx *ctx)
{
    if (!ctx->circuits)
        return;
    ctx->circuits->wave_choice.clear();   // wave times may have changed
    for (auto &kv : ctx->circuits->plans)
        if (kv.second->graph) {
            cudaGraphExecDestroy(kv.second->graph);
            kv.second->graph = nullptr;
        }
}

void release_circuits(tfhe_ctx *ctx)
{
    delete ctx->circuits;
    ctx->circuits = nullptr;
}

static std::string signature(const tfhe_job *jobs, size_t njobs)
{
    std::string key;
    char buf[96];
    for (size_t j = 0; j < njobs; ++j) {
        std::snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%lld;", jobs[j].kind, jobs[j].width,
                      jobs[j].rows, jobs[j].cols, (long long)jobs[j].batch);
        key += buf;
    }
    return key;
}

// Host-side schedule of a job list: pool layout, and every gate instance's
// level.  No device memory is touched.
struct Schedule {
    std::vector<JobLayout> jobs;
    long pool_rows = 0, gates = 0, max_width = 0, nout = 0;
    int depth = 0;
    std::vector<long> level_off;                 // depth + 1 entries
    std::vector<uint8_t> ops;                    // per scheduled gate, level-major
    std::vector<int32_t> ia, ib, ic, io, outs;
    bool three = false;                          // some gate has a third input
};

// Deadline-driven list scheduling (policy TFHE_SCHED_BALANCED): gate g of a
// netlist has ASAP level asap(g) and, for the schedule depth D, ALAP level
// alap(g) = D + 1 - height(g), height = longest path to an output.  Level L
// takes every ready gate whose deadline is L, then fills up to the next
// multiple of `target` (one GPU wave; at least one) with the ready gates of
// the earliest deadlines, so that no launch ends in a part-empty wave while
// work is ready.  By induction every gate is ready by its deadline, so the
// depth stays D; widths exceed one wave only where the deadlines force it.  The ciphertexts do not depend
// on the schedule (each gate is a deterministic function of its inputs).
static void balanced_levels(const std::vector<const Netlist *> &nets, const std::vector<long> &batch,
                            int D, long target, std::vector<std::vector<int32_t>> &level)
{
    const size_t nj = nets.size();
    std::vector<std::vector<int32_t>> alap(nj), cons_off(nj), cons(nj);
    std::vector<long> node_off(nj + 1, 0);
    for (size_t j = 0; j < nj; ++j) {
        const Netlist &nl = *nets[j];
        const int G = (int)nl.op.size();
        std::vector<int32_t> height(G, 1);
        for (int g = G - 1; g >= 0; --g)
            for (int in : {nl.a[g], nl.b[g], nl.c[g]})
                if (in >= nl.n_in)
                    height[in - nl.n_in] = std::max(height[in - nl.n_in], height[g] + 1);
        alap[j].resize(G);
        for (int g = 0; g < G; ++g)
            alap[j][g] = D + 1 - height[g];
        cons_off[j].assign(G + 1, 0);
        for (int g = 0; g < G; ++g)
            for (int in : {nl.a[g], nl.b[g], nl.c[g]})
                if (in >= nl.n_in)
                    cons_off[j][in - nl.n_in + 1]++;
        for (int g = 0; g < G; ++g)
            cons_off[j][g + 1] += cons_off[j][g];
        cons[j].resize(cons_off[j][G]);
        std::vector<int32_t> fillc(cons_off[j].begin(), cons_off[j].end() - 1);
        for (int g = 0; g < G; ++g)
            for (int in : {nl.a[g], nl.b[g], nl.c[g]})
                if (in >= nl.n_in)
                    cons[j][fillc[in - nl.n_in]++] = g;
        node_off[j + 1] = node_off[j] + batch[j] * G;
        level[j].assign((size_t)batch[j] * G, 0);
    }
    const long total = node_off[nj];
    std::vector<int32_t> pending(total);
    // ready buckets by deadline; a node is (job, instance, gate) packed in node id
    std::vector<std::vector<long>> bucket(D + 2);
    std::vector<size_t> head(D + 2, 0);
    auto job_of = [&](long node) {
        return (size_t)(std::upper_bound(node_off.begin(), node_off.end(), node) - node_off.begin() - 1);
    };
    for (size_t j = 0; j < nj; ++j) {
        const Netlist &nl = *nets[j];
        const int G = (int)nl.op.size();
        for (long inst = 0; inst < batch[j]; ++inst)
            for (int g = 0; g < G; ++g) {
                const long id = node_off[j] + inst * G + g;
                pending[id] = (nl.a[g] >= nl.n_in) + (nl.b[g] >= nl.n_in) + (nl.c[g] >= nl.n_in);
                if (pending[id] == 0)
                    bucket[alap[j][g]].push_back(id);
            }
    }
    long done = 0;
    std::vector<long> chosen, fresh;
    for (int L = 1; done < total; ++L) {
        chosen.clear();
        for (int a = 1; a <= L && a <= D; ++a) {   // deadline L (and, defensively, earlier)
            std::vector<long> &B = bucket[a];
            while (head[a] < B.size())
                chosen.push_back(B[head[a]++]);
        }
        // fill the last wave the forced gates leave open (at least one
        // wave) with the ready gates of the earliest deadlines
        const long cap = std::max(target, ((long)chosen.size() + target - 1) / target * target);
        for (int a = L + 1; a <= D && (long)chosen.size() < cap; ++a) {
            std::vector<long> &B = bucket[a];
            while (head[a] < B.size() && (long)chosen.size() < cap)
                chosen.push_back(B[head[a]++]);
        }
        fresh.clear();
        for (long id : chosen) {
            const size_t j = job_of(id);
            const Netlist &nl = *nets[j];
            const long G = (long)nl.op.size(), rel = id - node_off[j];
            const long inst = rel / G;
            const int g = (int)(rel % G);
            level[j][(size_t)rel] = L;
            for (int q = cons_off[j][g]; q < cons_off[j][g + 1]; ++q) {
                const long cid = node_off[j] + inst * G + cons[j][q];
                if (--pending[cid] == 0)
                    fresh.push_back(cid);
            }
        }
        for (long id : fresh) {
            const size_t j = job_of(id);
            const long G = (long)nets[j]->op.size();
            bucket[alap[j][(id - node_off[j]) % G]].push_back(id);
        }
        done += (long)chosen.size();
    }
}

static int build_schedule(tfhe_ctx *ctx, const tfhe_job *jobs, size_t njobs, int policy,
                          long target, Schedule &S)
{
    std::vector<const Netlist *> nets(njobs);
    std::vector<std::shared_ptr<const Netlist>> keep(njobs);
    std::vector<long> batch(njobs);
    long pool = 0, nout = 0;
    int depth = 0;
    for (size_t j = 0; j < njobs; ++j) {
        const tfhe_job &J = jobs[j];
        if (J.batch < 0)
            return fail(ctx, TFHE_EINVAL, "job %zu: negative batch", j);
        keep[j] = get_netlist(J.kind, J.width, J.rows, J.cols);
        if (!keep[j])
            return fail(ctx, TFHE_EINVAL, "job %zu: unsupported circuit (kind %d width %d)", j,
                        J.kind, J.width);
        nets[j] = keep[j].get();
        batch[j] = J.batch;
        JobLayout L;
        L.kind = J.kind;
        L.w = J.width;
        L.rows = J.rows;
        L.cols = J.cols;
        L.batch = J.batch;
        L.base = pool;
        L.inst_rows = nets[j]->wires();
        input_groups(J.kind, J.width, J.rows, J.cols, L.rows0, L.rows1);
        L.n_out = (long)nets[j]->out.size();
        L.out_off = nout;
        pool += L.inst_rows * J.batch;
        nout += L.n_out * J.batch;
        if (J.batch > 0)
            depth = std::max(depth, nets[j]->depth);
        S.jobs.push_back(L);
    }
    if (pool >= (1L << 31) / 2)
        return fail(ctx, TFHE_EINVAL, "batch too large for one schedule (%ld pool rows)", pool);
    // level of every gate instance
    std::vector<std::vector<int32_t>> level(njobs);
    if (policy == TFHE_SCHED_BALANCED && depth > 0) {
        balanced_levels(nets, batch, depth, std::max(target, 1L), level);
    } else {
        for (size_t j = 0; j < njobs; ++j) {
            level[j].resize((size_t)batch[j] * nets[j]->op.size());
            for (long inst = 0; inst < batch[j]; ++inst)
                std::copy(nets[j]->level.begin(), nets[j]->level.end(),
                          level[j].begin() + inst * nets[j]->op.size());
        }
    }
    int D = 0;
    for (auto &lv : level)
        for (int32_t l : lv)
            D = std::max(D, (int)l);
    std::vector<long> count(D + 2, 0);
    for (auto &lv : level)
        for (int32_t l : lv)
            count[l]++;
    S.level_off.assign(D + 1, 0);
    for (int l = 1; l <= D; ++l) {
        S.level_off[l] = S.level_off[l - 1] + count[l];
        S.max_width = std::max(S.max_width, count[l]);
    }
    const long total = D ? S.level_off[D] : 0;
    S.ops.resize(total);
    S.ia.resize(total);
    S.ib.resize(total);
    S.io.resize(total);
    for (size_t j = 0; j < njobs; ++j)
        S.three |= batch[j] > 0 && nets[j]->has3();
    if (S.three)
        S.ic.resize(total);
    S.outs.resize(nout);
    std::vector<long> fill(S.level_off.begin(), S.level_off.end());
    for (size_t j = 0; j < njobs; ++j) {
        const Netlist &nl = *nets[j];
        const JobLayout &L = S.jobs[j];
        const long G = (long)nl.op.size();
        for (long inst = 0; inst < L.batch; ++inst) {
            const long b = L.base + inst * L.inst_rows;
            for (long g = 0; g < G; ++g) {
                const long k = fill[level[j][inst * G + g] - 1]++;
                S.ops[k] = nl.op[g];
                S.ia[k] = (int32_t)(b + nl.a[g]);
                S.ib[k] = (int32_t)(b + nl.b[g]);
                if (S.three)
                    S.ic[k] = nl.c[g] >= 0 ? (int32_t)(b + nl.c[g]) : 0;
                S.io[k] = (int32_t)(b + nl.n_in + g);
            }
            for (size_t o = 0; o < nl.out.size(); ++o)
                S.outs[L.out_off + inst * L.n_out + o] = (int32_t)(b + nl.out[o]);
        }
    }
    S.pool_rows = pool;
    S.gates = total;
    S.depth = D;
    S.nout = nout;
    return TFHE_OK;
}

static int compile_plan(tfhe_ctx *ctx, const tfhe_job *jobs, size_t njobs, int policy,
                        long target, Plan &P)
{
    for (size_t j = 0; j < njobs; ++j)
        if (jobs[j].batch > 0 && (!jobs[j].in0 || !jobs[j].in1 || !jobs[j].out))
            return fail(ctx, TFHE_EINVAL, "job %zu: null pointer", j);
    Schedule S;
    int rc = build_schedule(ctx, jobs, njobs, policy, target, S);
    if (rc != TFHE_OK)
        return rc;
    P.jobs = S.jobs;
    P.pool_rows = S.pool_rows;
    P.gates = S.gates;
    P.max_width = S.max_width;
    P.depth = S.depth;
    P.level_off = S.level_off;
    P.h_ops = S.ops;
    const long total = S.gates, nout = S.nout, pool = S.pool_rows;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess && bytes)
            e = cudaMalloc(p, bytes);
    };
    alloc((void **)&P.pool, (size_t)std::max(pool, 1L) * kLweStride * sizeof(int32_t));
    alloc((void **)&P.big, (size_t)std::max(P.max_width, 1L) * kBigStride * sizeof(int32_t));
    alloc((void **)&P.d_ops, std::max(total, 1L));
    alloc((void **)&P.d_ia, std::max(total, 1L) * sizeof(int32_t));
    alloc((void **)&P.d_ib, std::max(total, 1L) * sizeof(int32_t));
    alloc((void **)&P.d_io, std::max(total, 1L) * sizeof(int32_t));
    if (S.three)
        alloc((void **)&P.d_ic, std::max(total, 1L) * sizeof(int32_t));
    alloc((void **)&P.d_out_rows, std::max(nout, 1L) * sizeof(int32_t));
    if (e == cudaSuccess && total) {
        e = cudaMemcpy(P.d_ops, S.ops.data(), total, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P.d_ia, S.ia.data(), total * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P.d_ib, S.ib.data(), total * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(P.d_io, S.io.data(), total * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && S.three)
            e = cudaMemcpy(P.d_ic, S.ic.data(), total * sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && nout)
        e = cudaMemcpy(P.d_out_rows, S.outs.data(), nout * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "compile schedule");
    return TFHE_OK;
}

// Level sequence: one blind-rotation and one key-switch launch per level.
// With profile set, events are recorded around both launches (as external
// event-record nodes when the stream is being captured).
static cudaError_t enqueue_levels(tfhe_ctx *ctx, Plan &P, cudaStream_t st, bool profile,
                                  bool capturing)
{
    if (profile && P.ev.empty()) {
        P.ev.resize(3 * (size_t)P.depth, nullptr);
        for (cudaEvent_t &e : P.ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess)
                return r;
        }
    }
    auto mark = [&](int idx) -> cudaError_t {
        if (!profile)
            return cudaSuccess;
        return capturing ? cudaEventRecordWithFlags(P.ev[idx], st, cudaEventRecordExternal)
                         : cudaEventRecord(P.ev[idx], st);
    };
    long kernels = 0;
    for (int l = 1; l <= P.depth; ++l) {
        const long off = P.level_off[l - 1], cnt = P.level_off[l] - off;
        if (cnt == 0)
            continue;
        cudaError_t e = mark(3 * (l - 1));
        DevKeys K = ctx->keys;
        if (P.wide_shape && K.br_group == 0 && cnt >= P.wave)
            K.br_group = P.wide_shape;
        if (e == cudaSuccess)
            e = launch_blind_rotate(K, P.d_ops + off, P.pool, P.d_ia + off, P.pool_rows,
                                    P.pool, P.d_ib + off, P.pool_rows, P.big, cnt, kMu,
                                    ctx->status, ctx->br_grid, st, P.d_ic ? P.pool : nullptr,
                                    P.d_ic ? P.d_ic + off : nullptr, P.pool_rows);
        if (e == cudaSuccess)
            e = mark(3 * (l - 1) + 1);
        if (e == cudaSuccess)
            e = launch_keyswitch(ctx->keys.ksk, P.big, P.pool, P.d_io + off, P.pool_rows, cnt,
                                 ctx->prm.n, ctx->num_sms, ctx->status, st, &ctx->keys);
        if (e == cudaSuccess)
            e = mark(3 * (l - 1) + 2);
        if (e != cudaSuccess)
            return e;
        kernels += 1 + keyswitch_kernels(cnt, ctx->num_sms, &ctx->keys);
    }
    P.kernels_per_run = kernels;
    return cudaSuccess;
}

// Baseline schedule: every gate on its own, one launch pair per gate.
static cudaError_t enqueue_per_gate(tfhe_ctx *ctx, Plan &P, cudaStream_t st)
{
    for (long k = 0; k < P.gates; ++k) {
        cudaError_t e = launch_blind_rotate(ctx->keys, P.d_ops + k, P.pool, P.d_ia + k, P.pool_rows,
                                            P.pool, P.d_ib + k, P.pool_rows, P.big, 1, kMu,
                                            ctx->status, ctx->br_grid, st,
                                            P.d_ic ? P.pool : nullptr,
                                            P.d_ic ? P.d_ic + k : nullptr, P.pool_rows);
        if (e != cudaSuccess)
            return e;
        e = launch_keyswitch(ctx->keys.ksk, P.big, P.pool, P.d_io + k, P.pool_rows, 1, ctx->prm.n,
                             ctx->num_sms, ctx->status, st, &ctx->keys);
        if (e != cudaSuccess)
            return e;
        ctx->launches += 1 + keyswitch_kernels(1, ctx->num_sms, &ctx->keys);
    }
    return cudaSuccess;
}

static int run_plan(tfhe_ctx *ctx, Plan &P, const tfhe_job *jobs, cudaStream_t st)
{
    NvtxRange range("tfhe: circuit schedule (levels of blind rotation + key switch)");
    CircuitCache &C = cache_of(ctx);
    cudaError_t e = cudaSuccess;
    // inputs -> pool (strided 2D copies, one per input group)
    for (size_t j = 0; j < P.jobs.size() && e == cudaSuccess; ++j) {
        const JobLayout &L = P.jobs[j];
        if (L.batch == 0)
            continue;
        const size_t row = kLweStride * sizeof(int32_t);
        e = cudaMemcpy2DAsync(P.pool + L.base * kLweStride, L.inst_rows * row, jobs[j].in0,
                              L.rows0 * row, L.rows0 * row, L.batch, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(P.pool + (L.base + L.rows0) * kLweStride, L.inst_rows * row,
                                  jobs[j].in1, L.rows1 * row, L.rows1 * row, L.batch,
                                  cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "copy inputs");
    if (C.per_gate) {
        e = enqueue_per_gate(ctx, P, st);
    } else if (C.use_graphs && !P.graph_failed) {
        if (P.graph && P.graph_profiled != C.profile) {   // recapture with/without events
            cudaGraphExecDestroy(P.graph);
            P.graph = nullptr;
        }
        if (!P.graph) {
            if (!C.capture_stream)
                e = cudaStreamCreateWithFlags(&C.capture_stream, cudaStreamNonBlocking);
            cudaGraph_t g = nullptr;
            if (e == cudaSuccess)
                e = cudaStreamBeginCapture(C.capture_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = enqueue_levels(ctx, P, C.capture_stream, C.profile, true);
                cudaError_t e2 = cudaStreamEndCapture(C.capture_stream, &g);
                e = e1 != cudaSuccess ? e1 : e2;
            }
            if (e == cudaSuccess)
                e = cudaGraphInstantiate(&P.graph, g, 0);
            if (g)
                cudaGraphDestroy(g);
            if (e != cudaSuccess) {  // fall back to direct launches for this plan
                (void)cudaGetLastError();
                P.graph = nullptr;
                P.graph_failed = true;
                e = cudaSuccess;
            }
            P.graph_profiled = C.profile;
        }
        if (P.graph) {
            e = cudaGraphLaunch(P.graph, st);
            ctx->launches += P.kernels_per_run;
        } else {
            e = enqueue_levels(ctx, P, st, C.profile, false);
            ctx->launches += P.kernels_per_run;
        }
    } else {
        e = enqueue_levels(ctx, P, st, C.profile, false);
        ctx->launches += P.kernels_per_run;
    }
    if (e == cudaSuccess && C.profile && !C.per_gate &&
        std::find(C.profiled.begin(), C.profiled.end(), &P) == C.profiled.end())
        C.profiled.push_back(&P);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "level launches");
    // pool -> outputs
    for (size_t j = 0; j < P.jobs.size() && e == cudaSuccess; ++j) {
        const JobLayout &L = P.jobs[j];
        const long cnt = L.n_out * L.batch;
        if (cnt == 0)
            continue;
        e = launch_gather_rows(jobs[j].out, P.pool, P.pool_rows, P.d_out_rows + L.out_off, cnt,
                               ctx->status, st);
        ctx->launches += 1;
    }
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "copy outputs");
    return TFHE_OK;
}

// Level unit of a job mix's schedule (the width the deadline scheduler
// rounds levels up to): one bootstrap per SM (levels run at the tuned
// narrow shape: lowest latency for a lone request), one wave of 4 per SM
// (the tuned shapes), or one wave of 5 per SM (levels of a wave or more at
// kBrFive).  Each candidate's schedule is costed with the autotuner's
// measurements: a level of w gates costs the measured time of its width
// bucket while w fits one 4-per-SM wave, ceil(w / wave) wave times above
// (at 5 per SM for the 5-per-SM candidate), and the cheapest schedule is
// used once it is at least 1 % cheaper than the 4-per-SM one.  Decided
// once per job mix; without autotuner measurements the unit is one wave of
// 4 per SM.
static long choose_wave(tfhe_ctx *ctx, CircuitCache &C, const std::string &sig,
                        const tfhe_job *jobs, size_t njobs)
{
    const long w1 = ctx->num_sms, w4 = 4L * ctx->num_sms, w5 = 5L * ctx->num_sms;
    const DevKeys &K = ctx->keys;
    const float t4 = K.wave_ms[0], t5 = K.wave_ms[1];
    if (!(t4 > 0.f))
        return w4;
    auto it = C.wave_choice.find(sig);
    if (it != C.wave_choice.end())
        return it->second;
    auto level_cost = [&](long n, long unit) -> double {
        if (unit == w5 && n >= w5)
            return (double)((n + w5 - 1) / w5) * t5;
        if (n > w4)
            return (double)((n + w4 - 1) / w4) * t4;
        const int b = tune_bucket(n);
        return K.tune_ms[b] > 0.f ? K.tune_ms[b] : t4;
    };
    auto cost = [&](long unit) -> double {
        Schedule S;
        if (build_schedule(nullptr, jobs, njobs, TFHE_SCHED_BALANCED, unit, S) != TFHE_OK)
            return -1.0;
        double c = 0;
        for (int l = 1; l <= S.depth; ++l)
            c += level_cost(S.level_off[l] - S.level_off[l - 1], unit);
        return c;
    };
    const double c4 = cost(w4);
    long pick = w4;
    double best = c4;
    if (c4 >= 0) {
        if (K.tune_ms[0] > 0.f && w1 <= kTuneEdge[0]) {
            const double c1 = cost(w1);
            if (c1 >= 0 && c1 < 0.99 * best)
                pick = w1, best = c1;
        }
        if (t5 > 0.f && t5 / w5 < 0.99f * t4 / w4) {
            const double c5 = cost(w5);
            if (c5 >= 0 && c5 < 0.99 * best)
                pick = w5, best = c5;
        }
    }
    C.wave_choice[sig] = pick;
    return pick;
}

int run_jobs(tfhe_ctx *ctx, const tfhe_job *jobs, size_t njobs, cudaStream_t st)
{
    if (!ctx->keys_loaded)
        return fail(ctx, TFHE_EINVAL, "keys not set");
    if (njobs == 0)
        return TFHE_OK;
    CircuitCache &C = cache_of(ctx);
    const std::string sig = signature(jobs, njobs);
    long target = C.level_width > 0 ? C.level_width : 4L * ctx->num_sms;
    if (C.level_width == 0 && C.policy == TFHE_SCHED_BALANCED)
        target = choose_wave(ctx, C, sig, jobs, njobs);
    const int wide = target == 5L * ctx->num_sms && C.level_width == 0 ? kBrFive : 0;
    const std::string key = sig + "|" + std::to_string(C.policy) + ":" + std::to_string(target);
    auto it = C.plans.find(key);
    if (it == C.plans.end()) {
        std::unique_ptr<Plan> P(new Plan());
        int rc = compile_plan(ctx, jobs, njobs, C.policy, target, *P);
        if (rc != TFHE_OK)
            return rc;
        if (C.order.size() >= 32) {   // keep device memory bounded
            Plan *victim = C.plans[C.order.front()].get();
            C.profiled.erase(std::remove(C.profiled.begin(), C.profiled.end(), victim),
                             C.profiled.end());
            C.plans.erase(C.order.front());
            C.order.erase(C.order.begin());
        }
        P->wave = target;
        P->wide_shape = wide;
        C.order.push_back(key);
        it = C.plans.emplace(key, std::move(P)).first;
    }
    return run_plan(ctx, *it->second, jobs, st);
}

}  // namespace tgb

using namespace tgb;

extern "C" {

int tfhe_run_jobs(tfhe_ctx *ctx, const tfhe_job *jobs, size_t njobs, void *stream)
{
    if (!ctx || (njobs && !jobs))
        return ctx ? fail(ctx, TFHE_EINVAL, "tfhe_run_jobs: null argument") : TFHE_EINVAL;
    DeviceGuard dg(ctx->device);
    return run_jobs(ctx, jobs, njobs, (cudaStream_t)stream);
}

static int one_job(tfhe_ctx *ctx, int kind, int width, int rows, int cols, const int32_t *a,
                   const int32_t *b, int32_t *out, size_t batch, void *stream)
{
    if (!ctx)
        return TFHE_EINVAL;
    if (batch == 0)
        return TFHE_OK;
    tfhe_job J;
    J.kind = kind;
    J.width = width;
    J.rows = rows;
    J.cols = cols;
    J.batch = (int64_t)batch;
    J.in0 = a;
    J.in1 = b;
    J.out = out;
    return tfhe_run_jobs(ctx, &J, 1, stream);
}

int tfhe_add_n(tfhe_ctx *ctx, int width, const int32_t *A, const int32_t *B, int32_t *R,
               size_t batch, void *stream)
{
    return one_job(ctx, TFHE_CIRCUIT_ADD, width, 0, 0, A, B, R, batch, stream);
}

int tfhe_mul_n(tfhe_ctx *ctx, int width, const int32_t *A, const int32_t *B, int32_t *R,
               size_t batch, void *stream)
{
    return one_job(ctx, TFHE_CIRCUIT_MUL, width, 0, 0, A, B, R, batch, stream);
}

int tfhe_matvec(tfhe_ctx *ctx, int width, int rows, int cols, const int32_t *M, const int32_t *v,
                int32_t *y, void *stream)
{
    return one_job(ctx, TFHE_CIRCUIT_MATVEC, width, rows, cols, M, v, y, 1, stream);
}

int tfhe_schedule_info(const tfhe_job *jobs, size_t njobs, int policy, int64_t target,
                       int32_t *widths, int32_t cap, int32_t *depth, int64_t *gates)
{
    if ((njobs && !jobs) || target < 0)
        return TFHE_EINVAL;
    Schedule S;
    int rc = build_schedule(nullptr, jobs, njobs, policy, target > 0 ? (long)target : 608L, S);
    if (rc != TFHE_OK)
        return rc;
    if (depth)
        *depth = S.depth;
    if (gates)
        *gates = S.gates;
    if (widths)
        for (int l = 1; l <= S.depth && l <= cap; ++l)
            widths[l - 1] = (int32_t)(S.level_off[l] - S.level_off[l - 1]);
    return TFHE_OK;
}

int tfhe_circuit_info(int kind, int width, int rows, int cols, int64_t *gates, int32_t *depth)
{
    Netlist nl;
    if (!build_netlist(kind, width, rows, cols, nl))
        return TFHE_EINVAL;
    if (gates)
        *gates = (int64_t)nl.op.size();
    if (depth)
        *depth = nl.depth;
    return TFHE_OK;
}

int tfhe_circuit_eval_plain(int kind, int width, int rows, int cols, const uint8_t *in,
                            size_t n_in, uint8_t *out, size_t n_out)
{
    const std::shared_ptr<const Netlist> keep = get_netlist(kind, width, rows, cols);
    if (!keep)
        return TFHE_EINVAL;
    const Netlist &nl = *keep;
    if (!in || !out || n_in != (size_t)nl.n_in || n_out != nl.out.size())
        return TFHE_EINVAL;
    std::vector<uint8_t> v(nl.wires());
    for (int i = 0; i < nl.n_in; ++i)
        v[i] = in[i] & 1u;
    for (size_t g = 0; g < nl.op.size(); ++g) {
        const int a = v[nl.a[g]], b = v[nl.b[g]], c = nl.c[g] >= 0 ? v[nl.c[g]] : 0;
        int r;
        switch (nl.op[g]) {
        case TFHE_NAND:  r = !(a & b); break;
        case TFHE_AND:   r = a & b; break;
        case TFHE_OR:    r = a | b; break;
        case TFHE_XOR:   r = a ^ b; break;
        case TFHE_NOR:   r = !(a | b); break;
        case TFHE_XNOR:  r = !(a ^ b); break;
        case TFHE_MAJ:   r = (a + b + c) >= 2; break;
        case TFHE_ANDNY: r = !a & b; break;
        case TFHE_ANDYN: r = a & !b; break;
        case TFHE_ORNY:  r = !a | b; break;
        case TFHE_ORYN:  r = a | !b; break;
        default:         return TFHE_EINVAL;
        }
        v[nl.n_in + g] = (uint8_t)r;
    }
    for (size_t o = 0; o < nl.out.size(); ++o)
        out[o] = v[nl.out[o]];
    return TFHE_OK;
}

int tfhe_ctx_set_option(tfhe_ctx *ctx, int option, int64_t value)
{
    if (!ctx)
        return TFHE_EINVAL;
    CircuitCache &C = cache_of(ctx);
    switch (option) {
    case TFHE_OPT_GRAPHS:
        C.use_graphs = value != 0;
        return TFHE_OK;
    case TFHE_OPT_PER_GATE:
        C.per_gate = value != 0;
        return TFHE_OK;
    case TFHE_OPT_PROFILE:
        C.profile = value != 0;
        return TFHE_OK;
    case TFHE_OPT_SCHEDULE:
        if (value != TFHE_SCHED_ASAP && value != TFHE_SCHED_BALANCED)
            return fail(ctx, TFHE_EINVAL, "TFHE_OPT_SCHEDULE must be ASAP or BALANCED");
        C.policy = (int)value;
        return TFHE_OK;
    case TFHE_OPT_LEVEL_WIDTH:
        if (value < 0)
            return fail(ctx, TFHE_EINVAL, "TFHE_OPT_LEVEL_WIDTH must be >= 0");
        C.level_width = (long)value;
        return TFHE_OK;
    case TFHE_OPT_TEST_FREE_HBM:
        if (value < 0)
            return fail(ctx, TFHE_EINVAL, "TFHE_OPT_TEST_FREE_HBM must be >= 0");
        ctx->test_free_hbm = (size_t)value;
        return TFHE_OK;
    case TFHE_OPT_TEST_KS_STALL:
        ctx->keys.ks_stall = value != 0;
        invalidate_graphs(ctx);
        return TFHE_OK;
    case TFHE_OPT_KS_KERNEL:
        if (value != 0 && value != kKsTiled &&
            !(value >= 1 && value <= 32 && (value & (value - 1)) == 0))
            return fail(ctx, TFHE_EINVAL, "TFHE_OPT_KS_KERNEL must be 0, 64 or 1, 2, 4, .. 32");
        ctx->keys.ks_kernel = (int)value;
        invalidate_graphs(ctx);   // captured graphs hold the old launch shape
        return TFHE_OK;
    case TFHE_OPT_BR_GROUP:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != kBrSplit &&
            value != kBrPair && value != kBrStaged && value != kBrStagedCtl &&
            value != kBrSplitStaged && value != kBrFive && value != kBrPairStaged)
            return fail(ctx, TFHE_EINVAL, "TFHE_OPT_BR_GROUP must be 0, 1, 2, 4, 5, 8, 16, 32, 33, 40 or 48");
        ctx->keys.br_group = (int)value;
        invalidate_graphs(ctx);   // captured graphs hold the old launch shape
        return TFHE_OK;
    default:
        return fail(ctx, TFHE_EINVAL, "unknown option %d", option);
    }
}

int tfhe_ctx_profile(tfhe_ctx *ctx, double *br_ms, int64_t *br_launches, int64_t *br_bootstraps,
                     double *ks_ms, int64_t *ks_launches)
{
    if (!ctx)
        return TFHE_EINVAL;
    DeviceGuard dg(ctx->device);
    CircuitCache &C = cache_of(ctx);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tfhe_ctx_profile");
    double bt = 0, kt = 0;
    int64_t bl = 0, kl = 0, bb = 0;
    for (Plan *P : C.profiled) {
        for (int l = 1; l <= P->depth; ++l) {
            const long cnt = P->level_off[l] - P->level_off[l - 1];
            if (cnt == 0)
                continue;
            float a = 0, b = 0;
            if (cudaEventElapsedTime(&a, P->ev[3 * (l - 1)], P->ev[3 * (l - 1) + 1]) != cudaSuccess ||
                cudaEventElapsedTime(&b, P->ev[3 * (l - 1) + 1], P->ev[3 * (l - 1) + 2]) != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(ctx, TFHE_ECUDA, "profile events not recorded");
            }
            bt += a;
            kt += b;
            bl += 1;
            bb += cnt;
            kl += keyswitch_kernels(cnt, ctx->num_sms, &ctx->keys);
        }
    }
    C.profiled.clear();
    if (br_ms) *br_ms = bt;
    if (br_launches) *br_launches = bl;
    if (br_bootstraps) *br_bootstraps = bb;
    if (ks_ms) *ks_ms = kt;
    if (ks_launches) *ks_launches = kl;
    return TFHE_OK;
}

}  // extern "C"
