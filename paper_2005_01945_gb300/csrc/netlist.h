// netlist.h -- boolean circuits as gate lists with ASAP levels (host).
#pragma once
#include <algorithm>
#include <cstdint>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

namespace tgb {

struct Netlist {
    int n_in = 0;                    // wires [0, n_in) are inputs
    std::vector<uint8_t> op;         // gate g drives wire n_in + g
    std::vector<int32_t> a, b, c;    // input wires of every gate (c = -1: two inputs)
    std::vector<int32_t> out;        // output wires in output order
    std::vector<int32_t> level;      // ASAP level of every gate (>= 1)
    int depth = 0;

    int gate(int o, int x, int y, int z = -1)
    {
        op.push_back((uint8_t)o);
        a.push_back(x);
        b.push_back(y);
        c.push_back(z);
        return n_in + (int)op.size() - 1;
    }
    bool has3() const
    {
        for (int32_t z : c)
            if (z >= 0)
                return true;
        return false;
    }
    int wires() const { return n_in + (int)op.size(); }

    void levelise()
    {
        std::vector<int32_t> wl(wires(), 0);
        level.resize(op.size());
        depth = 0;
        for (size_t g = 0; g < op.size(); ++g) {
            const int l = 1 + std::max(std::max(wl[a[g]], wl[b[g]]), c[g] >= 0 ? wl[c[g]] : 0);
            level[g] = l;
            wl[n_in + g] = l;
            depth = std::max(depth, l);
        }
    }
};

// Builds the netlist of one instance of a circuit (kinds of tfhe_circuit).
// Input wires: ADD/MUL: A bits [0, w), B bits [w, 2w).  GATE: a = 0, b = 1.
// MATVEC: M[r][c] bits at (r*cols + c)*w + bit, then v[c] bits.
bool build_netlist(int kind, int w, int rows, int cols, Netlist &nl);

// Shared, immutable netlists (thread-safe cache); nullptr if unsupported.
std::shared_ptr<const Netlist> get_netlist(int kind, int w, int rows, int cols);

// Rows per instance of the two input groups.
void input_groups(int kind, int w, int rows, int cols, long &rows0, long &rows1);

// Copies count ciphertext rows src[rows[i]] -> dst[i].
// dst row r = src row rows[r]; an index outside [0, src_rows) sets
// kErrGather in *status and leaves dst row r unwritten.
cudaError_t launch_gather_rows(int32_t *dst, const int32_t *src, long src_rows,
                               const int32_t *rows, long count, uint32_t *status,
                               cudaStream_t st);

}  // namespace tgb
