// Host runtime of the gradsim C ABI: context, mesh construction, launch sets,
// checkpointed rollout and adjoint, batching.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <system_error>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gs_internal.h"
#include "gs_runtime.h"

namespace gs {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

// NVTX range for profilers (forward phase, adjoint phase, each segment);
// costs nothing when no profiler is attached
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

gs_status set_error(gs_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}
gs_status cuda_error(cudaError_t e, const char* what) {
    return set_error(GS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
void clear_error() { g_last_error.clear(); }

// ---------------------------------------------------------------------------
// memory through the context
// ---------------------------------------------------------------------------
gs_status Buf::alloc(gs_ctx* c, size_t nbytes, cudaStream_t s) {
    release(s);
    if (nbytes == 0) return GS_OK;
    // reserve first, so concurrent allocations cannot overshoot the budget together
    const size_t before = c->used.fetch_add(nbytes);
    if (c->budget && before + nbytes > c->budget) {
        c->used.fetch_sub(nbytes);
        return set_error(GS_ENOMEM, "allocation of " + std::to_string(nbytes) + " bytes exceeds the context budget");
    }
    void* q = nullptr;
    if (c->has_alloc) {
        q = c->alloc.alloc(nbytes, (void*)s, c->alloc.user);
        if (!q) {
            c->used.fetch_sub(nbytes);
            return set_error(GS_ENOMEM, "allocator callback returned NULL for " + std::to_string(nbytes) + " bytes");
        }
    } else {
        cudaError_t e = cudaMallocAsync(&q, nbytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->used.fetch_sub(nbytes);
            return set_error(GS_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        }
    }
    if (((uintptr_t)q & 255) != 0) {  // bulk copies need 16 B; the library assumes cudaMalloc's 256 B
        if (c->has_alloc) c->alloc.free(q, nbytes, (void*)s, c->alloc.user);
        else cudaFreeAsync(q, s);
        c->used.fetch_sub(nbytes);
        return set_error(GS_EINVAL, "device allocation is not 256-byte aligned");
    }
    ctx = c;
    p = q;
    bytes = nbytes;
    return GS_OK;
}

void Buf::release(cudaStream_t s) {
    if (!p) return;
    if (ctx->has_alloc) ctx->alloc.free(p, bytes, (void*)s, ctx->alloc.user);
    else cudaFreeAsync(p, s);
    ctx->used.fetch_sub(bytes);
    p = nullptr;
    bytes = 0;
}

template <class T>
static gs_status upload(gs_ctx* c, Buf& b, const std::vector<T>& v, cudaStream_t s) {
    GS_TRY(b.alloc(c, std::max<size_t>(v.size(), 1) * sizeof(T), s));
    if (!v.empty()) GS_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return GS_OK;
}

// ---------------------------------------------------------------------------
// mesh construction (host): ordering, patches, local CSR, boundary CSR
// ---------------------------------------------------------------------------
static uint64_t spread21(uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

struct Topology {
    std::vector<int> elem_perm, hinge_perm, node_perm, node_inv;
    std::vector<PatchDesc> patches;
    std::vector<uint2> eidx, hidx;
    std::vector<int> bnd_ids;
    std::vector<uint16_t> loc_rowptr, loc_slots;
    std::vector<int> bnd_rowptr, part_pos;
    std::vector<uint4> topo;  // per patch: row pointers, slots, partial positions (16 B aligned pieces)
    int n_int = 0, n_bnd = 0, max_loc = 0, max_slots = 0, max_rec = 0;
    size_t smem_fwd[2] = {0, 0}, smem_adj[2] = {0, 0};  // [without, with] the extra stage regions
};


// augmenting path for row r over the groups in avail[r] not yet seen (Kuhn)
static bool bank_augment(int r, const unsigned* avail, int* match_g, int* row_g, unsigned& seen) {
    unsigned m = avail[r] & ~seen;
    while (m) {
        const int g = __builtin_ctz(m);
        m &= m - 1;
        seen |= 1u << g;
        if (match_g[g] < 0 || bank_augment(match_g[g], avail, match_g, row_g, seen)) {
            match_g[g] = r;
            row_g[r] = g;
            return true;
        }
    }
    return false;
}

// Order the entries of each local CSR row (the node's corner slots) so that
// the rows the node phase reads together hit distinct shared-memory banks.
// The node phase gives local node l to consumer thread l (mod the thread
// count); a quarter-warp (8 consecutive nodes) issues each 16-byte corner
// load together, and those 8 loads are conflict-free when the slots lie in 8
// different 16-byte bank groups (slot mod 8).  Column by column, the quarter's
// rows are matched to bank groups: greedily (each row the first free group at
// or after its rotation), then by augmenting paths (Kuhn) for the rows left
// over.  The padding reads of exhausted rows (the zero slot, one address,
// shared by broadcast) keep their group.  The order of a node's terms is
// fixed by the mesh and the patching alone, so sums stay bitwise
// reproducible.  `fill[l]` is the end of row l's entries.
static void order_rows_for_banks(uint16_t* slots, const int* rc, const int* fill, int n_loc, uint16_t zero_slot) {
    constexpr int kQ = 8, kG = 8;
    const unsigned zbit = 1u << (zero_slot % kG);
    std::vector<uint16_t> ent;  // a quarter's entries, row by row, grouped by bank group
    for (int q0 = 0; q0 < n_loc; q0 += kQ) {
        const int nq = std::min(kQ, n_loc - q0);
        int len[kQ] = {0}, padded[kQ] = {0}, maxlen = 0;
        int next[kQ][kG], left[kQ][kG];
        unsigned avail[kQ] = {0};  // groups with entries left, per row
        size_t total = 0;
        for (int i = 0; i < nq; ++i) total += (size_t)(fill[q0 + i] - rc[q0 + i]);
        ent.resize(total);
        int at = 0;
        for (int i = 0; i < nq; ++i) {
            const int l = q0 + i;
            len[i] = fill[l] - rc[l];
            padded[i] = rc[l + 1] - rc[l];
            maxlen = std::max(maxlen, padded[i]);
            for (int g = 0; g < kG; ++g) left[i][g] = 0;
            for (int k = rc[l]; k < fill[l]; ++k) left[i][slots[k] % kG]++;
            int put[kG];
            for (int g = 0; g < kG; ++g) {
                next[i][g] = put[g] = at;
                at += left[i][g];
                if (left[i][g]) avail[i] |= 1u << g;
            }
            for (int k = rc[l]; k < fill[l]; ++k) ent[put[slots[k] % kG]++] = slots[k];
        }
        for (int col = 0; col < maxlen; ++col) {
            unsigned taken = 0;
            for (int i = 0; i < nq; ++i)
                if (col >= len[i] && col < padded[i]) taken = zbit;
            int match_g[kG], row_g[kQ];
            for (int g = 0; g < kG; ++g) match_g[g] = -1;
            // greedy first (each row its free group with the most entries left),
            // then augmenting paths for the rows left without one
            unsigned used = taken;
            for (int i = 0; i < nq; ++i) {
                row_g[i] = -1;
                const unsigned f = avail[i] & ~used & 0xffu;
                if (!f) continue;
                // the first free group at or after (i + col) mod 8
                const int w = (i + col) % kG;
                const unsigned rot = ((f >> w) | (f << (kG - w))) & 0xffu;
                const int g = (w + __builtin_ctz(rot)) % kG;
                used |= 1u << g;
                match_g[g] = i;
                row_g[i] = g;
            }
            // an augmenting path ends at a group that is free and that some row
            // can take; without one, the rows left over keep a conflict
            unsigned want = 0;
            for (int i = 0; i < nq; ++i) want |= avail[i];
            for (int i = 0; i < nq && (want & ~used & 0xffu); ++i) {
                if (!avail[i] || row_g[i] >= 0) continue;
                unsigned seen = taken;
                if (bank_augment(i, avail, match_g, row_g, seen)) {
                    used = taken;
                    for (int g = 0; g < kG; ++g)
                        if (match_g[g] >= 0) used |= 1u << g;
                }
            }
            for (int i = 0; i < nq; ++i) {
                if (!avail[i]) continue;
                int g = row_g[i];
                if (g < 0) {  // no free group: the one with the most entries left
                    g = __builtin_ctz(avail[i]);
                    for (unsigned m = avail[i]; m; m &= m - 1) {
                        const int h = __builtin_ctz(m);
                        if (left[i][h] > left[i][g]) g = h;
                    }
                }
                slots[rc[q0 + i] + col] = ent[next[i][g]++];
                if (--left[i][g] == 0) avail[i] &= ~(1u << g);
            }
        }
        for (int i = 0; i < nq; ++i)
            for (int k = len[i]; k < padded[i]; ++k) slots[rc[q0 + i] + k] = zero_slot;
    }
}

static gs_status build_topology(const gs_mesh_desc& d, int pe, Topology& T) {
    const int N = d.n_nodes, E = d.n_elems, B = d.kind == GS_CLOTH ? d.n_hinges : 0;
    const int nc = d.kind == GS_TET ? 4 : 3;
    // 1. Morton order of element centroids
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], d.X[3 * i + k]);
            hi[k] = std::max(hi[k], d.X[3 * i + k]);
        }
    double ext = 0.0;
    for (int k = 0; k < 3; ++k) ext = std::max(ext, hi[k] - lo[k]);
    if (!(ext > 0.0)) ext = 1.0;
    std::vector<std::pair<uint64_t, int>> key(E);
    for (int e = 0; e < E; ++e) {
        double c[3] = {0, 0, 0};
        for (int j = 0; j < nc; ++j)
            for (int k = 0; k < 3; ++k) c[k] += d.X[3 * d.elems[nc * e + j] + k];
        uint64_t q[3];
        for (int k = 0; k < 3; ++k) {
            const double t = (c[k] / nc - lo[k]) / ext;
            q[k] = (uint64_t)std::min(2097151.0, std::max(0.0, t * 2097151.0));
        }
        key[e] = {spread21(q[0]) | spread21(q[1]) << 1 | spread21(q[2]) << 2, e};
    }
    std::sort(key.begin(), key.end());
    T.elem_perm.resize(E);
    std::vector<int> elem_inv(E);
    for (int e = 0; e < E; ++e) {
        T.elem_perm[e] = key[e].second;
        elem_inv[key[e].second] = e;
    }
    const int P = (E + pe - 1) / pe;
    // 2. hinges follow the patch of the triangle (x1, x3, x4)
    std::vector<int> hinge_patch(B, 0);
    if (B) {
        std::unordered_map<uint64_t, int> tri_of;
        tri_of.reserve(2 * E);
        auto tkey = [](int a, int b, int c) {
            int v[3] = {a, b, c};
            std::sort(v, v + 3);
            return (uint64_t)v[0] * 0x9E3779B97F4A7C15ULL ^ ((uint64_t)v[1] << 21) ^ ((uint64_t)v[2] << 42);
        };
        for (int t = 0; t < E; ++t) tri_of[tkey(d.elems[3 * t], d.elems[3 * t + 1], d.elems[3 * t + 2])] = t;
        for (int h = 0; h < B; ++h) {
            const int* q = d.hinges + 4 * h;
            auto it = tri_of.find(tkey(q[0], q[2], q[3]));
            if (it == tri_of.end())
                return set_error(GS_EINVAL, "hinge " + std::to_string(h) + ": triangle (x1, x3, x4) is not in the mesh");
            hinge_patch[h] = elem_inv[it->second] / pe;
        }
        std::vector<std::pair<int, int>> hk(B);
        for (int h = 0; h < B; ++h) hk[h] = {hinge_patch[h], h};
        std::sort(hk.begin(), hk.end());
        T.hinge_perm.resize(B);
        for (int h = 0; h < B; ++h) T.hinge_perm[h] = hk[h].second;
    }
    // per patch element / hinge ranges
    T.patches.assign(P, PatchDesc{});
    for (int p = 0; p < P; ++p) {
        T.patches[p].e_begin = p * pe;
        T.patches[p].n_e = std::min(pe, E - p * pe);
    }
    for (int h = 0, p = 0; p < P; ++p) {
        T.patches[p].h_begin = h;
        while (h < B && hinge_patch[T.hinge_perm[h]] == p) ++h;
        T.patches[p].n_h = h - T.patches[p].h_begin;
    }
    // corner nodes of internal element e / hinge h (caller node ids)
    auto ecorner = [&](int e, int c) { return d.elems[nc * T.elem_perm[e] + c]; };
    auto hcorner = [&](int h, int c) { return d.hinges[4 * T.hinge_perm[h] + c]; };
    // 3. patches touching each node
    std::vector<int> cnt(N, 0), last(N, -1), first(N, -1);
    auto touch = [&](int p, int u) {
        if (last[u] != p) {
            last[u] = p;
            if (cnt[u]++ == 0) first[u] = p;
        }
    };
    for (int p = 0; p < P; ++p) {
        const PatchDesc& q = T.patches[p];
        for (int e = q.e_begin; e < q.e_begin + q.n_e; ++e)
            for (int c = 0; c < nc; ++c) touch(p, ecorner(e, c));
        for (int h = q.h_begin; h < q.h_begin + q.n_h; ++h)
            for (int c = 0; c < 4; ++c) touch(p, hcorner(h, c));
    }
    // 4. internal node numbering: interior nodes patch by patch, then boundary
    //    nodes by (first patch, id), then untouched nodes
    //    (each patch's interior nodes by descending corner count, so the
    //    threads of a warp walk CSR rows of similar length)
    std::vector<int> deg(N, 0);
    for (int e = 0; e < E; ++e)
        for (int c = 0; c < nc; ++c) deg[ecorner(e, c)]++;
    for (int h = 0; h < B; ++h)
        for (int c = 0; c < 4; ++c) deg[hcorner(h, c)]++;
    std::vector<std::vector<int>> interior(P);
    std::vector<std::pair<int, int>> bnodes;
    std::vector<int> loose;
    for (int u = 0; u < N; ++u) {
        if (cnt[u] == 1) interior[first[u]].push_back(u);
        else if (cnt[u] > 1) bnodes.push_back({first[u], u});
        else loose.push_back(u);
    }
    for (auto& v : interior)
        std::sort(v.begin(), v.end(), [&](int x, int y) { return deg[x] != deg[y] ? deg[x] > deg[y] : x < y; });
    std::sort(bnodes.begin(), bnodes.end());
    T.node_perm.clear();
    T.node_perm.reserve(N);
    for (int p = 0; p < P; ++p) {
        T.patches[p].int_begin = (int)T.node_perm.size();
        T.patches[p].n_int = (int)interior[p].size();
        for (int u : interior[p]) T.node_perm.push_back(u);
    }
    T.n_int = (int)T.node_perm.size();
    for (auto& b : bnodes) T.node_perm.push_back(b.second);
    for (int u : loose) T.node_perm.push_back(u);
    T.n_bnd = N - T.n_int;
    T.node_inv.assign(N, -1);
    for (int i = 0; i < N; ++i) T.node_inv[T.node_perm[i]] = i;
    // 5. per patch: boundary list, local indices, local CSR
    T.eidx.assign(E, make_uint2(0, 0));
    T.hidx.assign(B, make_uint2(0, 0));
    std::vector<int> loc(N, -1), pdeg(N, 0);
    std::vector<int> bcount(T.n_bnd, 0);   // partials per boundary node so far
    std::vector<int> entry_node, entry_j;  // per (patch, boundary local node)
    for (int p = 0; p < P; ++p) {
        PatchDesc& q = T.patches[p];
        std::vector<int> bl;  // internal ids of boundary nodes touched by p
        auto note = [&](int u) {
            const int g = T.node_inv[u];
            if (g >= T.n_int) {
                if (loc[g] == -1) {
                    loc[g] = -2;
                    bl.push_back(g);
                }
                pdeg[g]++;
            }
        };
        for (int e = q.e_begin; e < q.e_begin + q.n_e; ++e)
            for (int c = 0; c < nc; ++c) note(ecorner(e, c));
        for (int h = q.h_begin; h < q.h_begin + q.n_h; ++h)
            for (int c = 0; c < 4; ++c) note(hcorner(h, c));
        // descending corner count within the patch (similar row lengths per warp)
        std::sort(bl.begin(), bl.end(), [&](int x, int y) { return pdeg[x] != pdeg[y] ? pdeg[x] > pdeg[y] : x < y; });
        // each patch's list starts 16 B aligned (its partial positions are bulk-copied)
        while (T.bnd_ids.size() % 4) {
            T.bnd_ids.push_back(0);
            entry_node.push_back(-1);
            entry_j.push_back(0);
        }
        q.bnd_begin = (int)T.bnd_ids.size();
        q.n_bnd = (int)bl.size();
        for (int k = 0; k < q.n_bnd; ++k) {
            loc[bl[k]] = q.n_int + k;
            T.bnd_ids.push_back(bl[k]);
            const int b = bl[k] - T.n_int;
            entry_node.push_back(b);
            entry_j.push_back(bcount[b]++);
        }
        for (int l = 0; l < q.n_int; ++l) loc[q.int_begin + l] = l;
        const int n_loc = q.n_int + q.n_bnd;
        const int n_rec = q.n_e + q.n_h;
        if (n_loc > 65535 || 4 * n_rec + 1 > 65535)
            return set_error(GS_EINVAL, "patch too large for 16-bit local indices; lower patch_elems");
        auto lid = [&](int u) { return (uint32_t)loc[T.node_inv[u]]; };
        // local ids, and the CSR over corner codes (record << 2 | corner) in
        // ascending code order (= ascending element order, hinges last; step 7
        // reorders each row against bank conflicts); the stored slot is the
        // corner's float4 index in the staged record planes, corner * n_rec +
        // record, and rows are padded to a multiple of 4 with index 4 * n_rec
        // (a zero float4 after the planes)
        std::vector<int> rc(n_loc + 1, 0);
        std::vector<std::pair<int, int>> code_node;  // (code, local node)
        code_node.reserve(nc * q.n_e + 4 * q.n_h);
        for (int le = 0; le < q.n_e; ++le) {
            const int e = q.e_begin + le;
            uint32_t l[4] = {0, 0, 0, 0};
            for (int c = 0; c < nc; ++c) {
                l[c] = lid(ecorner(e, c));
                code_node.push_back({4 * le + c, (int)l[c]});
            }
            T.eidx[e] = make_uint2(l[0] | l[1] << 16, l[2] | l[3] << 16);
        }
        for (int lh = 0; lh < q.n_h; ++lh) {
            const int h = q.h_begin + lh;
            uint32_t l[4];
            for (int c = 0; c < 4; ++c) {
                l[c] = lid(hcorner(h, c));
                code_node.push_back({4 * (q.n_e + lh) + c, (int)l[c]});
            }
            T.hidx[h] = make_uint2(l[0] | l[1] << 16, l[2] | l[3] << 16);
        }
        for (auto& cn : code_node) rc[cn.second + 1]++;
        for (int l = 0; l < n_loc; ++l) rc[l + 1] = (rc[l + 1] + 3) / 4 * 4;  // padded row lengths
        for (int l = 0; l < n_loc; ++l) rc[l + 1] += rc[l];
        const int n_slots = rc[n_loc];
        if (n_slots > 65535) return set_error(GS_EINVAL, "patch has too many corners; lower patch_elems");
        q.n_slots = n_slots;
        // 16 B aligned starts for the bulk copies
        while (T.loc_rowptr.size() % 8) T.loc_rowptr.push_back(0);
        while (T.loc_slots.size() % 8) T.loc_slots.push_back(0);
        q.lr_begin = (int)T.loc_rowptr.size();
        q.slot_begin = (int)T.loc_slots.size();
        for (int l = 0; l <= n_loc; ++l) T.loc_rowptr.push_back((uint16_t)rc[l]);
        std::vector<uint16_t> slots(n_slots, (uint16_t)(4 * n_rec));
        std::vector<int> fill(rc.begin(), rc.end() - 1);
        // staged planes: elements [4][n_e], then hinges [4][n_h]
        auto slot_of = [&](int code) {
            const int r = code >> 2, c = code & 3;
            return r < q.n_e ? c * q.n_e + r : 4 * q.n_e + c * q.n_h + (r - q.n_e);
        };
        for (auto& cn : code_node) slots[fill[cn.second]++] = (uint16_t)slot_of(cn.first);
        T.loc_slots.insert(T.loc_slots.end(), slots.begin(), slots.end());
        T.max_loc = std::max(T.max_loc, n_loc);
        T.max_slots = std::max(T.max_slots, n_slots);
        T.max_rec = std::max(T.max_rec, n_rec);
        for (int x = 0; x < 2; ++x) {
            T.smem_fwd[x] =
                std::max(T.smem_fwd[x], patch_smem_bytes(d.kind, q.n_e, q.n_h, n_loc, q.n_int, n_slots, false, x != 0));
            T.smem_adj[x] =
                std::max(T.smem_adj[x], patch_smem_bytes(d.kind, q.n_e, q.n_h, n_loc, q.n_int, n_slots, true, x != 0));
        }
        for (int g : bl) {
            loc[g] = -1;
            pdeg[g] = 0;
        }
        for (int l = 0; l < q.n_int; ++l) loc[q.int_begin + l] = -1;
        q.mesh = 0;
    }
    // tail padding so a rounded-up bulk copy of the last patch stays in bounds
    for (int k = 0; k < 16; ++k) {
        T.loc_rowptr.push_back(0);
        T.loc_slots.push_back(0);
    }
    // 6. boundary CSR: node b's partials at [bnd_rowptr[b], bnd_rowptr[b+1]),
    //    in patch order; each (patch, boundary local node) knows its position
    T.bnd_rowptr.assign(T.n_bnd + 1, 0);
    for (int b = 0; b < T.n_bnd; ++b) T.bnd_rowptr[b + 1] = T.bnd_rowptr[b] + bcount[b];
    // (padding entries point at partial 0 and are never used; 4 entries of
    // tail padding keep a rounded-up copy of the last list in bounds)
    T.part_pos.assign(entry_node.size() + 4, 0);
    for (size_t i = 0; i < entry_node.size(); ++i)
        if (entry_node[i] >= 0) T.part_pos[i] = T.bnd_rowptr[entry_node[i]] + entry_j[i];
    for (int k = 0; k < 4; ++k) T.bnd_ids.push_back(0);
    // 7. each patch's CSR rows ordered against bank conflicts (patches in
    // parallel: they are independent), then the topology blocks
    {
        // a worker that fails (host memory) records it; the pass then fails as
        // a whole once every thread has been joined
        std::atomic<bool> failed{false};
        auto order_range = [&](int p0, int p1) {
            std::vector<int> fill;
            for (int p = p0; p < p1; ++p) {
                const PatchDesc& q = T.patches[p];
                const int n_loc = q.n_int + q.n_bnd;
                const uint16_t zero = (uint16_t)(4 * (q.n_e + q.n_h));
                const uint16_t* rp = &T.loc_rowptr[q.lr_begin];
                uint16_t* sl = &T.loc_slots[q.slot_begin];
                std::vector<int> rc(rp, rp + n_loc + 1);
                fill.resize(n_loc);
                for (int l = 0; l < n_loc; ++l) {
                    int k = rc[l];
                    while (k < rc[l + 1] && sl[k] != zero) ++k;
                    fill[l] = k;
                }
                order_rows_for_banks(sl, rc.data(), fill.data(), n_loc, zero);
            }
        };
        auto order_patches = [&](int p0, int p1) {
            try {
                order_range(p0, p1);
            } catch (...) {
                failed = true;
            }
        };
        const int n_thr = std::max(1, std::min({(int)std::thread::hardware_concurrency(), 16, P / 256}));
        // patches [0, done) are handed to threads; if a thread cannot be
        // started, this thread orders the rest itself
        int done = 0;
        std::vector<std::thread> pool;
        pool.reserve(n_thr);
        for (int t = 1; t < n_thr; ++t) {
            const int p0 = (int)((long long)P * (t - 1) / n_thr), p1 = (int)((long long)P * t / n_thr);
            try {
                pool.emplace_back(order_patches, p0, p1);
            } catch (...) {  // std::system_error: no thread could be started
                break;
            }
            done = p1;
        }
        order_patches(done, P);
        for (auto& th : pool) th.join();
        if (failed) throw std::bad_alloc();
    }
    // per patch topology blocks for the one-copy staging
    auto append = [&](const void* src, size_t bytes) {
        const size_t n16 = (bytes + 15) / 16, at = T.topo.size();
        T.topo.resize(at + n16, make_uint4(0, 0, 0, 0));
        if (bytes) std::memcpy(&T.topo[at], src, bytes);
    };
    for (PatchDesc& q : T.patches) {
        const int n_loc = q.n_int + q.n_bnd;
        q.topo = (int)T.topo.size();
        append(&T.loc_rowptr[q.lr_begin], 2 * (size_t)(n_loc + 1));
        append(&T.loc_slots[q.slot_begin], 2 * (size_t)q.n_slots);
        append(&T.part_pos[q.bnd_begin], 4 * (size_t)q.n_bnd);
    }
    return GS_OK;
}

static std::vector<NodeBlock> make_blocks(int begin, int n, int per, int mesh) {
    std::vector<NodeBlock> v;
    for (int i = 0; i < n; i += per) v.push_back(NodeBlock{mesh, begin + i, std::min(per, n - i), 0});
    return v;
}

// explicit stability estimate (warning only): elastic dt < 2/omega with
// omega^2 ~ (lambda + 2 mu) V |Dm^-1|_F^2 / m_corner, contact and damping
// limits dt < 2/sqrt(k_e/m), dt < 2 m / k_d, dt < 2 m / k_f
static double stability_estimate(const gs_mesh_desc& d) {
    const int N = d.n_nodes, E = d.n_elems, nc = d.kind == GS_TET ? 4 : 3;
    std::vector<double> m(N, 0.0), V(E, 0.0), G(E, 0.0);
    for (int e = 0; e < E; ++e) {
        const int* q = d.elems + nc * e;
        double a[3], b[3], c[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = d.X[3 * q[1] + k] - d.X[3 * q[0] + k];
            b[k] = d.X[3 * q[2] + k] - d.X[3 * q[0] + k];
            c[k] = nc == 4 ? d.X[3 * q[3] + k] - d.X[3 * q[0] + k] : 0.0;
        }
        double la = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double lb = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        double lc = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        double h = nc == 4 ? std::min(la, std::min(lb, lc)) : std::min(la, lb);
        double n0 = a[1] * b[2] - a[2] * b[1], n1 = a[2] * b[0] - a[0] * b[2], n2 = a[0] * b[1] - a[1] * b[0];
        if (nc == 4) V[e] = std::fabs(n0 * c[0] + n1 * c[1] + n2 * c[2]) / 6.0;
        else V[e] = 0.5 * std::sqrt(n0 * n0 + n1 * n1 + n2 * n2);
        G[e] = (h > 0) ? 3.0 / (h * h) : 0.0;
        const double share = d.density[e] * V[e] / nc;
        for (int j = 0; j < nc; ++j) m[q[j]] += share;
    }
    double om2 = 0.0, mmin = 1e300;
    for (int e = 0; e < E; ++e) {
        const int* q = d.elems + nc * e;
        double me = 1e300;
        for (int j = 0; j < nc; ++j)
            if (!(d.pinned && d.pinned[q[j]])) me = std::min(me, m[q[j]]);
        if (me >= 1e300 || me <= 0) continue;
        om2 = std::max(om2, (d.lambda[e] + 2 * d.mu[e]) * V[e] * G[e] * 4.0 / me);
    }
    for (int i = 0; i < N; ++i)
        if (m[i] > 0 && !(d.pinned && d.pinned[i])) mmin = std::min(mmin, m[i]);
    double dt = om2 > 0 ? 2.0 / std::sqrt(om2) : 1e300;
    if (mmin < 1e300 && (d.contact.plane_on || d.contact.sphere_on)) {
        if (d.contact.ke > 0) dt = std::min(dt, 2.0 / std::sqrt(d.contact.ke / mmin));
        if (d.contact.kd > 0) dt = std::min(dt, 2.0 * mmin / d.contact.kd);
        if (d.contact.kf > 0) dt = std::min(dt, 2.0 * mmin / d.contact.kf);
    }
    return dt;
}

static bool finite_all(const double* p, int n) {
    if (!p) return true;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

static gs_status validate(const gs_mesh_desc& d) {
    if (d.kind != GS_TET && d.kind != GS_CLOTH) return set_error(GS_EINVAL, "kind must be GS_TET or GS_CLOTH");
    if (d.n_nodes <= 0 || d.n_elems <= 0) return set_error(GS_EINVAL, "mesh needs nodes and elements");
    if (!d.elems || !d.X || !d.mu || !d.lambda || !d.density) return set_error(GS_EINVAL, "missing mesh array");
    const int nc = d.kind == GS_TET ? 4 : 3;
    for (int e = 0; e < d.n_elems; ++e) {
        const int* q = d.elems + nc * e;
        for (int j = 0; j < nc; ++j) {
            if (q[j] < 0 || q[j] >= d.n_nodes)
                return set_error(GS_EINVAL, "element " + std::to_string(e) + " has node index out of range");
            for (int k = 0; k < j; ++k)
                if (q[k] == q[j]) return set_error(GS_EINVAL, "element " + std::to_string(e) + " repeats a node");
        }
        if (!(d.mu[e] > 0) || !(d.lambda[e] > 0) || !(d.density[e] > 0) || !std::isfinite(d.mu[e]) ||
            !std::isfinite(d.lambda[e]) || !std::isfinite(d.density[e]))
            return set_error(GS_EINVAL, "element " + std::to_string(e) + ": mu, lambda, density must be finite and > 0");
    }
    if (d.kind == GS_CLOTH) {
        if (d.n_hinges < 0 || (d.n_hinges > 0 && (!d.hinges || !d.kb)))
            return set_error(GS_EINVAL, "cloth hinges need indices and kb");
        for (int h = 0; h < d.n_hinges; ++h) {
            const int* q = d.hinges + 4 * h;
            for (int j = 0; j < 4; ++j)
                if (q[j] < 0 || q[j] >= d.n_nodes)
                    return set_error(GS_EINVAL, "hinge " + std::to_string(h) + " has node index out of range");
            if (!std::isfinite(d.kb[h])) return set_error(GS_EINVAL, "non-finite kb");
        }
        if (!finite_all(d.hinge_act, d.n_hinges)) return set_error(GS_EINVAL, "non-finite hinge actuation");
    }
    if (!finite_all(d.X, 3 * d.n_nodes) || !finite_all(d.v0, 3 * d.n_nodes) || !finite_all(d.act, d.n_elems))
        return set_error(GS_EINVAL, "non-finite positions, velocities or actuation");
    const gs_contact& c = d.contact;
    if (c.plane_on) {
        const double n = std::sqrt((double)c.plane_n[0] * c.plane_n[0] + (double)c.plane_n[1] * c.plane_n[1] +
                                   (double)c.plane_n[2] * c.plane_n[2]);
        if (std::fabs(n - 1.0) > 1e-5) return set_error(GS_EINVAL, "plane normal must have unit length");
    }
    if (c.sphere_on && !(c.sphere_r > 0)) return set_error(GS_EINVAL, "sphere radius must be > 0");
    if (!(c.ke >= 0 && c.kd >= 0 && c.kf >= 0 && c.mu_f >= 0)) return set_error(GS_EINVAL, "contact parameters must be >= 0");
    return GS_OK;
}

}  // namespace gs

using namespace gs;

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
gs_status gs_mesh::refresh_rt() {
    MeshRT& r = rt;
    r.st_x = (float4*)st.p;
    r.st_v = st.p ? (float4*)st.p + (size_t)n_bufs * n_pad : nullptr;
    r.st_f = st.p ? (float4*)st.p + 2 * (size_t)n_bufs * n_pad : nullptr;
    r.buf_stride = n_pad;
    r.xb = (float4*)xb.p;
    r.vb = (float4*)vb.p;
    r.wbar = (double*)wbar.p;
    r.g_ml = (double2*)g_ml.p;
    r.g_act = (double*)g_act.p;
    r.g_kb = (double*)g_kb.p;
    r.g_hact = (double*)g_hact.p;
    return GS_OK;
}

// grow the state block to hold `n` buffers, keeping buffer 0
gs_status gs_mesh::ensure_buffers(int n, cudaStream_t s) {
    if (n <= n_bufs && st.p) return GS_OK;
    Buf nb;
    GS_TRY(nb.alloc(ctx, (size_t)3 * n * n_pad * sizeof(float4), s));  // x, v, element forces
    if (st.p) {
        GS_CUDA(cudaMemcpyAsync(nb.p, st.p, (size_t)n_pad * sizeof(float4), cudaMemcpyDeviceToDevice, s));
        GS_CUDA(cudaMemcpyAsync((float4*)nb.p + (size_t)n * n_pad, (float4*)st.p + (size_t)n_bufs * n_pad,
                                (size_t)n_pad * sizeof(float4), cudaMemcpyDeviceToDevice, s));
    }
    st.release(s);
    st = std::move(nb);
    n_bufs = n;
    return refresh_rt();
}

gs_status gs_mesh::ensure_adjoint(cudaStream_t s) {
    if (xb.p) return GS_OK;
    GS_TRY(xb.alloc(ctx, (size_t)n_pad * sizeof(float4), s));
    GS_TRY(vb.alloc(ctx, (size_t)n_pad * sizeof(float4), s));
    GS_TRY(wbar.alloc(ctx, (size_t)n_pad * sizeof(double), s));
    GS_TRY(mbar.alloc(ctx, (size_t)n_pad * sizeof(double), s));
    // +2: tail padding for the rounded-up bulk copy of the last patch
    GS_TRY(g_ml.alloc(ctx, ((size_t)info.n_elems + 1) * sizeof(double2), s));
    GS_TRY(g_act.alloc(ctx, (size_t)info.n_elems * sizeof(double), s));
    if (info.n_hinges) {
        GS_TRY(g_kb.alloc(ctx, (size_t)info.n_hinges * sizeof(double), s));
        GS_TRY(g_hact.alloc(ctx, (size_t)info.n_hinges * sizeof(double), s));
    }
    return refresh_rt();
}

gs_mesh::~gs_mesh() {
    cudaStream_t s = 0;
    for (Buf* b : {&rec, &hrec, &Xs, &Xp, &v0, &bnd_ids, &loc_rowptr, &loc_slots, &bnd_rowptr,
                   &part_pos, &partials, &node_perm, &elem_perm, &hinge_perm, &w, &X, &rho, &pinned, &st, &xb, &vb,
                   &wbar, &mbar, &g_ml, &g_act, &g_kb, &g_hact, &status, &target, &scratch})
        b->release(s);
    self.reset();
    cudaStreamSynchronize(s);
}

extern "C" gs_status gs_mesh_create(gs_ctx* ctx, const gs_mesh_desc* desc, gs_mesh** out) try {
    clear_error();
    if (!ctx || !desc || !out) return set_error(GS_EINVAL, "null argument");
    *out = nullptr;
    return gs::mesh_create(ctx, desc, 0, out);
} GS_ABI_CATCH

static gs_status mesh_create_impl(gs_ctx* ctx, const gs_mesh_desc* desc, cudaStream_t s, gs_mesh** out);

// Builds a mesh with all its uploads and set-up kernels on stream s and waits
// for them; the mesh is ready for use on any stream when this returns.  The
// host-side build (ordering, patches, topology) allocates host memory: a
// failed allocation returns GS_ENOMEM (what was allocated is released) and
// never reaches the C caller, or a server's builder thread, as an exception.
gs_status gs::mesh_create(gs_ctx* ctx, const gs_mesh_desc* desc, cudaStream_t s, gs_mesh** out) {
    try {
        return mesh_create_impl(ctx, desc, s, out);
    } catch (const std::bad_alloc&) {
        return set_error(GS_ENOMEM, "host allocation failed while building the mesh");
    }
}

static gs_status mesh_create_impl(gs_ctx* ctx, const gs_mesh_desc* desc, cudaStream_t s, gs_mesh** out) {
    GS_CUDA(cudaSetDevice(ctx->device));
    const gs_mesh_desc& d = *desc;
    GS_TRY(validate(d));
    int threads = d.block_threads > 0 ? d.block_threads : 128;
    if (threads % 32 || threads > 1024) return set_error(GS_EINVAL, "block_threads must be a multiple of 32, <= 1024");
    const int threads_adj = d.block_threads_adj > 0 ? d.block_threads_adj : threads;
    if (threads_adj % 32 || threads_adj > 1024)
        return set_error(GS_EINVAL, "block_threads_adj must be a multiple of 32, <= 1024");
    int pe = d.patch_elems > 0 ? d.patch_elems : (d.kind == GS_TET ? 256 : 256);
    pe = (pe + 1) & ~1;  // even, so every patch's FP64 accumulators start 16 B aligned
    if (pe > 16383) return set_error(GS_EINVAL, "patch_elems must be <= 16383");
    Topology T;
    GS_TRY(build_topology(d, pe, T));
    std::unique_ptr<gs_mesh> m(new gs_mesh());
    m->ctx = ctx;
    const int N = d.n_nodes, E = d.n_elems, B = d.kind == GS_CLOTH ? d.n_hinges : 0;
    m->info.kind = d.kind;
    m->info.n_nodes = N;
    m->info.n_elems = E;
    m->info.n_hinges = B;
    m->info.n_patches = (int)T.patches.size();
    m->info.n_boundary_nodes = T.n_bnd;
    m->info.patch_elems = pe;
    m->info.block_threads = threads;
    m->info.block_threads_adj = threads_adj;
    m->info.dt_stable = stability_estimate(d);
    m->n_pad = (N + 31) & ~31;
    m->threads = threads;
    m->threads_adj = threads_adj;
    m->max_loc = T.max_loc;
    m->max_slots = T.max_slots;
    m->max_rec = T.max_rec;
    for (int x = 0; x < 2; ++x) {
        m->smem_fwd[x] = T.smem_fwd[x];
        m->smem_adj[x] = T.smem_adj[x];
    }
    m->patches = T.patches;
    m->bnd_blocks = make_blocks(0, T.n_bnd, kNodeBlock, 0);
    m->node_blocks = make_blocks(0, N, 256, 0);
    const size_t need = std::max(patch_dyn_smem((int)T.smem_adj[1]), sizeof(double) * (3 * (size_t)T.max_loc + 4 * (size_t)T.max_rec + 1));
    if (need > ctx->smem_optin)
        return set_error(GS_EINVAL, "patch needs " + std::to_string(need) + " B of shared memory; lower patch_elems");
    // element records in internal order, 4 planes (geometry filled by the set-up kernel)
    std::vector<float4> rec(4 * (size_t)E, make_float4(0.f, 0.f, 0.f, 0.f));
    std::vector<float> rho(E);
    auto bits = [](uint32_t u) {
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    };
    for (int e = 0; e < E; ++e) {
        const int u = T.elem_perm[e];
        rho[e] = (float)d.density[u];
        const float act = d.act ? (float)d.act[u] : 0.0f;
        if (d.kind == GS_TET) {
            rec[rec_at(E, pe, 2, e)] = make_float4(0.f, 0.f, (float)d.mu[u], (float)d.lambda[u]);
            rec[rec_at(E, pe, 3, e)] = make_float4(bits(T.eidx[e].x), bits(T.eidx[e].y), act, 0.f);
        } else {
            rec[rec_at(E, pe, 1, e)] = make_float4(0.f, (float)d.mu[u], (float)d.lambda[u], act);
            rec[rec_at(E, pe, 3, e)] = make_float4(bits(T.eidx[e].x), bits(T.eidx[e].y), 0.f, 0.f);
        }
    }
    std::vector<float4> hrec(4 * (size_t)B, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int h = 0; h < B; ++h) {
        const int u = T.hinge_perm[h];
        hrec[h].w = (float)d.kb[u];
        hrec[(size_t)B + h].w = d.hinge_act ? (float)d.hinge_act[u] : 0.0f;
        hrec[3 * (size_t)B + h] = make_float4(bits(T.hidx[h].x), bits(T.hidx[h].y), 0.f, 0.f);
    }
    std::vector<double> X(3 * (size_t)N);
    // contact offsets of the rest positions, formed in FP64
    std::vector<float4> Xs(N);
    std::vector<float> Xp(N);
    std::vector<float> v0(3 * (size_t)N, 0.0f);
    std::vector<uint8_t> pin(N, 0);
    for (int i = 0; i < N; ++i) {
        const int u = T.node_perm[i];
        for (int k = 0; k < 3; ++k) X[3 * (size_t)i + k] = d.X[3 * (size_t)u + k];
        const double* xi = &X[3 * (size_t)i];
        double dc[3], q = 0.0, np = 0.0;
        for (int k = 0; k < 3; ++k) {
            dc[k] = xi[k] - (double)d.contact.sphere_c[k];
            q += dc[k] * dc[k];
            np += (double)d.contact.plane_n[k] * xi[k];
        }
        q -= (double)d.contact.sphere_r * (double)d.contact.sphere_r;
        Xs[i] = make_float4((float)dc[0], (float)dc[1], (float)dc[2], (float)q);
        Xp[i] = (float)((double)d.contact.plane_h - np);
        pin[i] = d.pinned ? d.pinned[u] : 0;
    }
    // initial velocities in caller order (the state is set through the caller-order kernel)
    if (d.v0)
        for (size_t k = 0; k < 3 * (size_t)N; ++k) v0[k] = (float)d.v0[k];
    GS_TRY(upload(ctx, m->rec, rec, s));
    GS_TRY(upload(ctx, m->hrec, hrec, s));
    GS_TRY(upload(ctx, m->Xs, Xs, s));
    GS_TRY(upload(ctx, m->Xp, Xp, s));
    GS_TRY(upload(ctx, m->v0, v0, s));
    GS_TRY(upload(ctx, m->bnd_ids, T.bnd_ids, s));
    GS_TRY(upload(ctx, m->loc_rowptr, T.loc_rowptr, s));
    GS_TRY(upload(ctx, m->loc_slots, T.loc_slots, s));
    GS_TRY(upload(ctx, m->bnd_rowptr, T.bnd_rowptr, s));
    GS_TRY(upload(ctx, m->part_pos, T.part_pos, s));
    GS_TRY(upload(ctx, m->topo, T.topo, s));
    GS_TRY(m->partials.alloc(ctx, std::max<size_t>(T.bnd_ids.size(), 1) * sizeof(float4), s));
    GS_TRY(upload(ctx, m->node_perm, T.node_perm, s));
    GS_TRY(upload(ctx, m->elem_perm, T.elem_perm, s));
    GS_TRY(upload(ctx, m->hinge_perm, T.hinge_perm, s));
    GS_TRY(m->w.alloc(ctx, (size_t)m->n_pad * sizeof(float), s));
    GS_TRY(upload(ctx, m->X, X, s));
    GS_TRY(upload(ctx, m->rho, rho, s));
    GS_TRY(upload(ctx, m->pinned, pin, s));
    GS_TRY(m->status.alloc(ctx, 4 * sizeof(int), s));
    GS_CUDA(cudaMemsetAsync(m->status.p, 0, 4 * sizeof(int), s));
    GS_TRY(m->ensure_buffers(1, s));
    GS_CUDA(cudaMemsetAsync(m->st.p, 0, m->st.bytes, s));
    // runtime record
    MeshRT& r = m->rt;
    std::memset(&r, 0, sizeof(r));
    r.kind = d.kind;
    r.n_nodes = N;
    r.n_int = T.n_int;
    r.n_bnd = T.n_bnd;
    r.n_elems = E;
    r.n_hinges = B;
    r.act_ld = (E + 3) & ~3;  // 16 B rows: a patch's slice of a row is one bulk copy
    r.hact_ld = (B + 3) & ~3;
    r.active = ACT_FWD | ACT_ADJ;
    r.rec = (float4*)m->rec.p;
    r.hrec = (float4*)m->hrec.p;
    r.Xs = (const float4*)m->Xs.p;
    r.Xp = (const float*)m->Xp.p;
    r.Xd = (const double*)m->X.p;
    r.bnd_ids = (const int*)m->bnd_ids.p;
    r.loc_rowptr = (const uint16_t*)m->loc_rowptr.p;
    r.loc_slots = (const uint16_t*)m->loc_slots.p;
    r.topo = (const uint4*)m->topo.p;
    r.pe = pe;
    r.bnd_rowptr = (const int*)m->bnd_rowptr.p;
    r.n_part = T.bnd_rowptr.empty() ? 0 : T.bnd_rowptr[T.n_bnd];
    r.part_pos = (const int*)m->part_pos.p;
    r.partials = (float4*)m->partials.p;
    r.node_perm = (const int*)m->node_perm.p;
    r.elem_perm = (const int*)m->elem_perm.p;
    r.hinge_perm = (const int*)m->hinge_perm.p;
    r.w = (float*)m->w.p;
    r.ck_tick = -1;
    r.gx = d.gravity[0];
    r.gy = d.gravity[1];
    r.gz = d.gravity[2];
    r.ke = d.contact.ke;
    r.kd = d.contact.kd;
    r.kf = d.contact.kf;
    r.mu_f = d.contact.mu_f;
    r.plane_on = d.contact.plane_on;
    r.pnx = d.contact.plane_n[0];
    r.pny = d.contact.plane_n[1];
    r.pnz = d.contact.plane_n[2];
    r.ph = d.contact.plane_h;
    r.sphere_on = d.contact.sphere_on;
    r.scx = d.contact.sphere_c[0];
    r.scy = d.contact.sphere_c[1];
    r.scz = d.contact.sphere_c[2];
    r.sr = d.contact.sphere_r;
    r.status = (int*)m->status.p;
    m->refresh_rt();
    // the mesh's own launch set (its device MeshRT record)
    m->self.reset(new LaunchSet());
    GS_TRY(m->self->build(ctx, std::vector<gs_mesh*>{m.get()}, s));
    // a1 set-up on the GPU: Dm^-1, V / A, masses, inverse masses
    GS_TRY(m->run_setup(1, s));
    // initial state: u = 0 (x = X exactly), v = v0
    launch_reset_state(m->rt_dev(), (const float*)m->v0.p, s);
    int bad = 0;
    GS_CUDA(cudaMemcpyAsync(&bad, (int*)m->status.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    GS_CUDA(cudaGetLastError());
    if (bad) return set_error(GS_EINVAL, "inverted or degenerate rest element (non-positive volume or area)");
    m->info.device_bytes = 0;
    for (Buf* b : {&m->rec, &m->hrec, &m->Xs, &m->Xp, &m->v0, &m->bnd_ids, &m->loc_rowptr,
                   &m->loc_slots, &m->bnd_rowptr, &m->part_pos, &m->topo, &m->partials, &m->node_perm, &m->elem_perm,
                   &m->hinge_perm, &m->w, &m->X, &m->rho, &m->pinned, &m->st})
        m->info.device_bytes += b->bytes;
    *out = m.release();
    return GS_OK;
}

gs_status gs_mesh::run_setup(int geometry, cudaStream_t s) {
    Buf mass, part;
    GS_TRY(mass.alloc(ctx, (size_t)n_pad * sizeof(double), s));
    GS_TRY(part.alloc(ctx, std::max<size_t>(bnd_ids.bytes / sizeof(int), 1) * sizeof(double), s));
    const size_t sm = sizeof(double) * (3 * (size_t)max_loc + 4 * (size_t)max_rec + 1);
    launch_setup_mesh(self->launch, (const double*)X.p, (const float*)rho.p, (double*)mass.p, (double*)part.p,
                      (const uint8_t*)pinned.p, (int*)status.p + 1, geometry, sm, s);
    GS_CUDA(cudaGetLastError());
    mass.release(s);
    part.release(s);
    return GS_OK;
}

extern "C" void gs_mesh_destroy(gs_mesh* m) { delete m; }

extern "C" gs_status gs_mesh_info_get(const gs_mesh* m, gs_mesh_info* out) try {
    if (!m || !out) return set_error(GS_EINVAL, "null argument");
    *out = m->info;
    return GS_OK;
} GS_ABI_CATCH

// copy a caller buffer to a device scratch when it lives on the host
static gs_status stage_in(gs_ctx* ctx, Buf& tmp, const float* src, size_t n, int mem, cudaStream_t s,
                          const float** dev) {
    if (!src) {
        *dev = nullptr;
        return GS_OK;
    }
    if (mem == GS_MEM_DEVICE) {
        *dev = src;
        return GS_OK;
    }
    GS_TRY(tmp.alloc(ctx, n * sizeof(float), s));
    GS_CUDA(cudaMemcpyAsync(tmp.p, src, n * sizeof(float), cudaMemcpyHostToDevice, s));
    *dev = (const float*)tmp.p;
    return GS_OK;
}

extern "C" gs_status gs_mesh_set_params(gs_mesh* m, const float* mu, const float* lambda, const float* density,
                                        const float* act, const float* kb, int mem, void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t E = m->info.n_elems, B = m->info.n_hinges;
    Buf t1, t2, t3, t4, t5;
    const float *dmu = nullptr, *dlam = nullptr, *drho = nullptr, *dact = nullptr, *dkb = nullptr;
    GS_TRY(stage_in(m->ctx, t1, mu, E, mem, s, &dmu));
    GS_TRY(stage_in(m->ctx, t2, lambda, E, mem, s, &dlam));
    GS_TRY(stage_in(m->ctx, t3, density, E, mem, s, &drho));
    GS_TRY(stage_in(m->ctx, t4, act, E, mem, s, &dact));
    GS_TRY(stage_in(m->ctx, t5, kb, B, mem, s, &dkb));
    GS_TRY(m->self->sync_rt(s));
    if (dmu || dlam || dact || dkb) launch_scatter_params(m->rt_dev(), dmu, dlam, dact, dkb, s);
    if (drho) {
        // density -> internal order, then the lumped-mass set-up
        launch_gather_elems(m->rt_dev(), drho, (float*)m->rho.p, s);
        GS_TRY(m->run_setup(0, s));
    }
    m->ro.valid = false;
    GS_CUDA(cudaGetLastError());
    for (Buf* b : {&t1, &t2, &t3, &t4, &t5}) b->release(s);
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_mesh_set_state(gs_mesh* m, const float* x, const float* v, int mem, void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = 3 * (size_t)m->info.n_nodes;
    Buf t1, t2;
    const float *dx = nullptr, *dv = nullptr;
    GS_TRY(stage_in(m->ctx, t1, x, n, mem, s, &dx));
    GS_TRY(stage_in(m->ctx, t2, v, n, mem, s, &dv));
    GS_TRY(m->self->sync_rt(s));
    launch_set_state(m->rt_dev(), 0, dx, dv, s);
    GS_CUDA(cudaGetLastError());
    t1.release(s);
    t2.release(s);
    m->ro.valid = false;
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_mesh_reset(gs_mesh* m, void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    cudaStream_t s = (cudaStream_t)stream;
    GS_TRY(m->self->sync_rt(s));
    launch_reset_state(m->rt_dev(), (const float*)m->v0.p, s);
    GS_CUDA(cudaGetLastError());
    m->ro.valid = false;
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_mesh_get_state(gs_mesh* m, float* x, float* v, int mem, void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = 3 * (size_t)m->info.n_nodes;
    GS_TRY(m->self->sync_rt(s));
    if (mem == GS_MEM_DEVICE) {
        launch_get_state(m->rt_dev(), 0, x, v, s);
        GS_CUDA(cudaGetLastError());
        return GS_OK;
    }
    Buf t;
    GS_TRY(t.alloc(m->ctx, 2 * n * sizeof(float), s));
    launch_get_state(m->rt_dev(), 0, x ? (float*)t.p : nullptr, v ? (float*)t.p + n : nullptr, s);
    if (x) GS_CUDA(cudaMemcpyAsync(x, t.p, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (v) GS_CUDA(cudaMemcpyAsync(v, (float*)t.p + n, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    t.release(s);
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_mesh_check(gs_mesh* m, int reset, void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    GS_CUDA(cudaMemcpyAsync(&st, m->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (reset) GS_CUDA(cudaMemsetAsync(m->status.p, 0, sizeof(int), s));
    if (st & 4) return set_error(GS_EINDEX, "an index check of the checked build failed; results are invalid");
    if (st & 2) return set_error(GS_ETIMEOUT, "a bounded wait in a step kernel ran out; results are invalid");
    if (st & 1) return set_error(GS_ENONFINITE, "non-finite state");
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_selftest_bounded_wait(int iterations, int* status_out, void* stream) try {
    clear_error();
    if (!status_out || iterations < 1 || iterations > 1000000)
        return set_error(GS_EINVAL, "gs_selftest_bounded_wait: iterations in 1..1e6 and status_out required");
    return selftest_bounded_wait(iterations, status_out, (cudaStream_t)stream);
} GS_ABI_CATCH

// ---------------------------------------------------------------------------
// launch sets
// ---------------------------------------------------------------------------
gs_status LaunchSet::build(gs_ctx* c, const std::vector<gs_mesh*>& ms, cudaStream_t s) {
    ctx = c;
    meshes = ms;
    std::vector<PatchDesc> tp, cp;
    std::vector<NodeBlock> bb, nb;
    size_t sf_t[2] = {0, 0}, sa_t[2] = {0, 0}, sf_c[2] = {0, 0}, sa_c[2] = {0, 0};
    threads = 32;
    threads_adj = 32;
    node_block_begin.clear();
    for (int i = 0; i < (int)ms.size(); ++i) {
        gs_mesh* m = ms[i];
        auto& dst = m->info.kind == GS_TET ? tp : cp;
        for (PatchDesc p : m->patches) {
            p.mesh = i;
            dst.push_back(p);
        }
        for (NodeBlock b : m->bnd_blocks) {
            b.mesh = i;
            bb.push_back(b);
        }
        node_block_begin.push_back((int)nb.size());
        for (NodeBlock b : m->node_blocks) {
            b.mesh = i;
            nb.push_back(b);
        }
        for (int x = 0; x < 2; ++x) {
            if (m->info.kind == GS_TET) {
                sf_t[x] = std::max(sf_t[x], m->smem_fwd[x]);
                sa_t[x] = std::max(sa_t[x], m->smem_adj[x]);
            } else {
                sf_c[x] = std::max(sf_c[x], m->smem_fwd[x]);
                sa_c[x] = std::max(sa_c[x], m->smem_adj[x]);
            }
        }
        threads = std::max(threads, m->threads);
        threads_adj = std::max(threads_adj, m->threads_adj);
    }
    node_block_begin.push_back((int)nb.size());
    GS_TRY(upload(c, d_tet, tp, s));
    GS_TRY(upload(c, d_cloth, cp, s));
    GS_TRY(upload(c, d_bnd, bb, s));
    GS_TRY(upload(c, d_nodes, nb, s));
    GS_TRY(d_rt.alloc(c, std::max<size_t>(ms.size(), 1) * sizeof(MeshRT), s));
    GS_TRY(d_loss.alloc(c, std::max<size_t>(nb.size(), 1) * sizeof(double), s));
    host_rt.resize(ms.size());
    launch.tet_patches = (const PatchDesc*)d_tet.p;
    launch.n_tet_patches = (int)tp.size();
    launch.cloth_patches = (const PatchDesc*)d_cloth.p;
    launch.n_cloth_patches = (int)cp.size();
    launch.bnd_blocks = (const NodeBlock*)d_bnd.p;
    launch.n_bnd_blocks = (int)bb.size();
    launch.node_blocks = (const NodeBlock*)d_nodes.p;
    launch.n_node_blocks = (int)nb.size();
    launch.rt = (MeshRT*)d_rt.p;
    launch.threads = threads;
    launch.threads_adj = threads_adj;
    for (int x = 0; x < 2; ++x) {
        stage_var[x][0] = (int)sf_t[x];
        stage_var[x][1] = (int)sf_c[x];
        stage_var[x][2] = (int)sa_t[x];
        stage_var[x][3] = (int)sa_c[x];
    }
    launch.extras = -1;  // stages and grids set by sync_rt
    launch.bgrid[0] = boundary_grid(0, (int)bb.size(), c->num_sms);
    launch.bgrid[1] = boundary_grid(1, (int)bb.size(), c->num_sms);
    return sync_rt(s);
}

gs_status LaunchSet::sync_rt(cudaStream_t s) {
    launch.air = 0;
    int extras = 0;
    for (size_t i = 0; i < meshes.size(); ++i) {
        host_rt[i] = meshes[i]->rt;
        const MeshRT& r = host_rt[i];
        if (r.kind == GS_CLOTH && r.air_on) launch.air = 1;
        if (r.act_seq || r.hact_seq || (r.kind == GS_CLOTH && r.air_on)) extras = 1;
    }
    if (extras != launch.extras) {
        // stages with / without the actuation slices and boundary v; the grids follow their size
        launch.extras = extras;
        const int np[4] = {launch.n_tet_patches, launch.n_cloth_patches, launch.n_tet_patches, launch.n_cloth_patches};
        for (int k = 0; k < 4; ++k) {
            launch.stage[k] = stage_var[extras][k];
            const int thr = k < 2 ? launch.threads : launch.threads_adj;  // forward, adjoint kernels
            launch.grid[k] = patch_grid(k, thr, launch.stage[k], np[k], ctx->num_sms);
        }
    }
    GS_CUDA(cudaMemcpyAsync(d_rt.p, host_rt.data(), host_rt.size() * sizeof(MeshRT), cudaMemcpyHostToDevice, s));
    return GS_OK;
}

LaunchSet::~LaunchSet() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    for (Buf* b : {&d_tet, &d_cloth, &d_bnd, &d_nodes, &d_rt, &d_loss}) b->release(0);
}

// `steps` forward (phase 0) or adjoint (phase 1) steps, ticks 0..steps-1
gs_status LaunchSet::run(int phase, int steps, cudaStream_t s) {
    if (steps <= 0) return GS_OK;
    if (ctx->graphs && ctx->prof) {
        // timed launches in the graph path: a graph captured for this call
        // with an event node before and after every kernel (the event nodes
        // end the programmatic overlap between neighbouring kernels)
        cudaStream_t cs = ctx->capture_stream;
        GS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        ctx->prof->capture = true;
        for (int t = 0; t < steps; ++t) {
            if (phase == 0) launch_forward_step(launch, t, cs, ctx->prof);
            else launch_adjoint_step(launch, t, cs, ctx->prof);
        }
        ctx->prof->capture = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        e = cudaGraphLaunch(ge, s);
        cudaGraphExecDestroy(ge);  // freed once the launch completes
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
        return GS_OK;
    }
    if (!ctx->graphs) {
        for (int t = 0; t < steps; ++t) {
            if (phase == 0) launch_forward_step(launch, t, s, ctx->prof);
            else launch_adjoint_step(launch, t, s, ctx->prof);
        }
        GS_CUDA(cudaGetLastError());
        return GS_OK;
    }
    // the air adds a kernel to adjoint steps; the extra stage regions change stages and grids
    const std::pair<int, int> key{phase + 2 * launch.air + 4 * launch.extras, steps};
    auto it = graphs.find(key);
    if (it == graphs.end()) {
        cudaStream_t cs = ctx->capture_stream;
        GS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        for (int t = 0; t < steps; ++t) {
            if (phase == 0) launch_forward_step(launch, t, cs);
            else launch_adjoint_step(launch, t, cs);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        it = graphs.emplace(key, ge).first;
    }
    GS_CUDA(cudaGraphLaunch(it->second, s));
    return GS_OK;
}

static int choose_K(int S, int K) {
    if (K > 0) return std::min(K, std::max(S, 1));
    int k = (int)std::ceil(std::sqrt((double)std::max(S, 1)));
    return std::max(1, k);
}

// forward rollout over a launch set (App. B, checkpoint every K steps)
gs_status LaunchSet::rollout(const std::vector<float>& dts, int S, int K, const std::vector<const float*>& targets,
                             double* loss_dev, cudaStream_t s) {
    NvtxRange range("gs forward rollout");
    if (S < 0) return set_error(GS_EINVAL, "n_steps must be >= 0");
    K = choose_K(S, K);
    // K = 1 keeps every state (state n in buffer 1 + n): the adjoint then
    // needs no recomputation.  Otherwise checkpoints 1..n_ck hold the states
    // c K and K + 1 further buffers hold a recomputed segment.
    const bool all = K == 1;
    const int n_ck = std::max(1, (S + K - 1) / K);
    const int n_bufs = all ? S + 2 : 1 + n_ck + K + 1;
    gs_status warn = GS_OK;
    for (size_t i = 0; i < meshes.size(); ++i) {
        gs_mesh* m = meshes[i];
        if (!(dts[i] > 0.0f) || !std::isfinite(dts[i])) return set_error(GS_EINVAL, "dt must be finite and > 0");
        if (dts[i] > m->info.dt_stable) warn = GS_WUNSTABLE;
        GS_TRY(m->ensure_buffers(n_bufs, s));
        m->rt.dt = dts[i];
        m->ro.valid = false;
        if (targets[i]) {
            GS_TRY(m->target.alloc(ctx, 3 * (size_t)m->info.n_nodes * sizeof(float), s));
            GS_CUDA(cudaMemcpyAsync(m->target.p, targets[i], m->target.bytes, cudaMemcpyDeviceToDevice, s));
        } else {
            m->target.release(s);
        }
        m->rt.target = (const float*)m->target.p;
        m->rt.active = ACT_FWD | ACT_ADJ;
        // checkpoint 0 = the current state
        m->rt.cp_src = 0;
        m->rt.cp_dst = 1;
    }
    GS_TRY(sync_rt(s));
    launch_copy_state(launch, s);
    if (all) {
        // tick t reads buffer 1 + t and writes 2 + t; the final state is then
        // copied to buffer 0 (the current state)
        for (gs_mesh* m : meshes) {
            m->rt.in_a = 1;
            m->rt.in_b = 1;
            m->rt.out_a = 2;
            m->rt.out_b = 1;
            m->rt.ck_tick = -1;
            m->rt.st_a = 0;  // tick t is step t
            m->rt.st_b = 1;
        }
        GS_TRY(sync_rt(s));
        GS_TRY(run(0, S, s));
        for (gs_mesh* m : meshes) {
            m->rt.in_a = m->rt.in_b = m->rt.out_a = m->rt.out_b = 0;
            m->rt.cp_src = S + 1;
            m->rt.cp_dst = 0;
        }
        GS_TRY(sync_rt(s));
        launch_copy_state(launch, s);
    } else {
        for (int c = 0; c < n_ck; ++c) {
            NvtxRange seg("gs forward segment");
            const int steps = std::min(K, S - c * K);
            for (gs_mesh* m : meshes) {
                m->rt.in_a = m->rt.in_b = m->rt.out_a = m->rt.out_b = 0;
                m->rt.ck_tick = (c + 1 < n_ck) ? steps - 1 : -1;
                m->rt.ck_buf = 2 + c;
                m->rt.st_a = c * K;  // tick t is step c K + t
                m->rt.st_b = 1;
            }
            GS_TRY(sync_rt(s));
            GS_TRY(run(0, steps, s));
        }
    }
    for (gs_mesh* m : meshes) m->rt.ck_tick = -1;
    GS_TRY(sync_rt(s));
    if (loss_dev) {
        launch_seed_loss(launch, (double*)d_loss.p, 0, s);
        for (size_t i = 0; i < meshes.size(); ++i)
            launch_loss_finalize((const double*)d_loss.p, node_block_begin[i],
                                 node_block_begin[i + 1] - node_block_begin[i], loss_dev + i, s);
    }
    for (gs_mesh* m : meshes) {
        m->ro.valid = true;
        m->ro.S = S;
        m->ro.K = K;
        m->ro.n_ck = n_ck;
    }
    GS_CUDA(cudaGetLastError());
    return warn;
}

// discrete adjoint over the whole rollout: per segment (last first) restore
// the checkpoint, recompute and store the segment's states, then run the
// reverse steps (App. B).  A segment of n steps needs its states 0..n-1 and
// the element force at each, which the forward step from that state stores,
// so all n forward steps are recomputed; with every state kept (K = 1) the
// reverse steps read the stored states and forces directly.
gs_status LaunchSet::adjoint(const std::vector<const float*>& seed_x, const std::vector<const float*>& seed_v,
                             const std::vector<gs_grads>& grads, int keep, cudaStream_t s) {
    NvtxRange range("gs adjoint");
    for (gs_mesh* m : meshes)
        if (!m->ro.valid) return set_error(GS_ESTATE, "gs_adjoint needs a preceding gs_rollout");
    const int S = meshes[0]->ro.S, K = meshes[0]->ro.K, n_ck = meshes[0]->ro.n_ck;
    for (gs_mesh* m : meshes)
        if (m->ro.S != S || m->ro.K != K) return set_error(GS_ESTATE, "batch meshes have different rollouts");
    for (size_t i = 0; i < meshes.size(); ++i) {
        gs_mesh* m = meshes[i];
        GS_TRY(m->ensure_adjoint(s));
        m->rt.seed_x = seed_x[i];
        m->rt.seed_v = seed_v[i];
        // actuation gradients only when asked for (saves an FP64 read-modify-write per element-step)
        m->rt.g_act = grads[i].d_act ? (double*)m->g_act.p : nullptr;
        m->rt.g_hact = grads[i].d_hinge_act ? (double*)m->g_hact.p : nullptr;
        // per-step actuation gradients (internal order), every step written
        m->rt.d_act_seq = m->rt.d_hact_seq = nullptr;
        m->rt.n_dact = 0;
        if (grads[i].d_act_seq && S > 0) {
            GS_TRY(m->dact_seq.alloc(ctx, (size_t)S * m->rt.act_ld * sizeof(float), s));
            m->rt.d_act_seq = (float*)m->dact_seq.p;
            m->rt.n_dact = S;
        }
        if (grads[i].d_hinge_act_seq && S > 0 && m->info.n_hinges > 0) {
            GS_TRY(m->dhact_seq.alloc(ctx, (size_t)S * m->rt.hact_ld * sizeof(float), s));
            m->rt.d_hact_seq = (float*)m->dhact_seq.p;
            m->rt.n_dact = S;
        }
    }
    GS_TRY(sync_rt(s));
    launch_seed_loss(launch, (double*)d_loss.p, 1, s);
    launch_zero_adjoint(launch, s);
    for (gs_mesh* m : meshes) {
        launch_zero_f64((double*)m->g_ml.p, 2 * (long long)m->info.n_elems, s);
        if (m->rt.g_act) launch_zero_f64((double*)m->g_act.p, m->info.n_elems, s);
        launch_zero_f64((double*)m->g_kb.p, m->info.n_hinges, s);
        if (m->rt.g_hact) launch_zero_f64((double*)m->g_hact.p, m->info.n_hinges, s);
    }
    const int seg0 = 1 + n_ck;
    if (K == 1) {
        // tick t reverses step S-1-t, whose input state is in buffer S - t
        for (gs_mesh* m : meshes) {
            m->rt.ck_tick = -1;
            m->rt.adj_a = S;
            m->rt.adj_b = -1;
            m->rt.st_a = S - 1;
            m->rt.st_b = -1;
        }
        GS_TRY(sync_rt(s));
        GS_TRY(run(1, S, s));
    }
    for (int sg = K == 1 ? -1 : n_ck - 1; sg >= 0; --sg) {
        NvtxRange seg("gs adjoint segment (recompute + reverse)");
        const int steps = std::min(K, S - sg * K);
        for (gs_mesh* m : meshes) {
            MeshRT& r = m->rt;
            r.cp_src = 1 + sg;
            r.cp_dst = seg0;
            r.in_a = seg0;
            r.in_b = 1;
            r.out_a = seg0 + 1;
            r.out_b = 1;
            r.ck_tick = -1;
            r.adj_a = seg0 + steps - 1;
            r.adj_b = -1;
            r.st_a = sg * K;  // recompute: tick t is step sg K + t
            r.st_b = 1;
        }
        GS_TRY(sync_rt(s));
        launch_copy_state(launch, s);
        // all the segment's steps: the reverse steps read the states 0..n-1
        // and the element forces at each, which the forward step from that
        // state writes (the state after the last step is not read)
        GS_TRY(run(0, steps, s));
        for (gs_mesh* m : meshes) {
            m->rt.st_a = sg * K + steps - 1;  // reverse: tick t is step sg K + steps - 1 - t
            m->rt.st_b = -1;
        }
        GS_TRY(sync_rt(s));
        GS_TRY(run(1, steps, s));
    }
    for (size_t i = 0; i < meshes.size(); ++i) {
        gs_mesh* m = meshes[i];
        if (m->rt.d_act_seq)
            launch_permute_rows((const float*)m->dact_seq.p, grads[i].d_act_seq, S, m->info.n_elems, m->rt.act_ld,
                                (const int*)m->elem_perm.p, 0, s);
        if (m->rt.d_hact_seq)
            launch_permute_rows((const float*)m->dhact_seq.p, grads[i].d_hinge_act_seq, S, m->info.n_hinges,
                                m->rt.hact_ld, (const int*)m->hinge_perm.p, 0, s);
        m->rt.d_act_seq = m->rt.d_hact_seq = nullptr;
        m->rt.n_dact = 0;
        m->rt.seed_x = m->rt.seed_v = nullptr;
        const size_t sm = std::max(sizeof(double) * (size_t)m->max_loc, (size_t)16);
        GS_TRY(m->self->sync_rt(s));
        launch_finalize_grads(m->self->launch, (double*)m->mbar.p, grads[i], sm, s);
        if (!keep) m->ro.valid = false;
    }
    GS_TRY(sync_rt(s));
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status LaunchSet::step(const std::vector<float>& dts, int n, cudaStream_t s) {
    gs_status warn = GS_OK;
    for (size_t i = 0; i < meshes.size(); ++i) {
        gs_mesh* m = meshes[i];
        if (!(dts[i] > 0.0f) || !std::isfinite(dts[i])) return set_error(GS_EINVAL, "dt must be finite and > 0");
        if (dts[i] > m->info.dt_stable) warn = GS_WUNSTABLE;
        m->rt.dt = dts[i];
        m->rt.in_a = m->rt.in_b = m->rt.out_a = m->rt.out_b = 0;
        m->rt.ck_tick = -1;
        m->rt.active = ACT_FWD | ACT_ADJ;
        m->ro.valid = false;
    }
    const int chunk = 64;
    for (int done = 0; done < n; done += chunk) {
        for (gs_mesh* m : meshes) {
            m->rt.st_a = done;  // actuation rows done, done + 1, ...
            m->rt.st_b = 1;
        }
        GS_TRY(sync_rt(s));
        GS_TRY(run(0, std::min(chunk, n - done), s));
    }
    return warn;
}

// ---------------------------------------------------------------------------
// C ABI: library, context, single-mesh calls
// ---------------------------------------------------------------------------
extern "C" int gs_version(void) { return GS_VERSION; }
extern "C" const char* gs_last_error(void) { return g_last_error_cstr(); }

namespace gs {
const char* g_last_error_cstr() { return g_last_error.c_str(); }
}  // namespace gs

extern "C" gs_status gs_create(gs_ctx** out, int device, size_t budget, const gs_allocator* alloc) try {
    clear_error();
    if (!out) return set_error(GS_EINVAL, "null argument");
    *out = nullptr;
    int n = 0;
    GS_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return set_error(GS_EINVAL, "no such device");
    GS_CUDA(cudaSetDevice(device));
    std::unique_ptr<gs_ctx> c(new gs_ctx());
    c->device = device;
    c->budget = budget;
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    int optin = 0;
    GS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    GS_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    c->smem_optin = (size_t)optin;
    set_kernel_smem_limits(c->smem_optin);
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    *out = c.release();
    return GS_OK;
} GS_ABI_CATCH

cudaEvent_t EventProf::get() {
    if (pool.empty()) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
}
void EventProf::begin(int, cudaStream_t s) {
    open = get();
    if (capture) cudaEventRecordWithFlags(open, s, cudaEventRecordExternal);
    else cudaEventRecord(open, s);
}
void EventProf::end(int kind, cudaStream_t s) {
    cudaEvent_t b = get();
    if (capture) cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
    else cudaEventRecord(b, s);
    pending.push_back(Pending{kind, open, b});
    open = nullptr;
}
void EventProf::collect() {
    for (const Pending& p : pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            total_ms[p.kind] += ms;
            launches[p.kind] += 1;
        }
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.clear();
}
EventProf::~EventProf() {
    collect();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

extern "C" gs_status gs_profile(gs_ctx* c, int enable) try {
    clear_error();
    if (!c) return set_error(GS_EINVAL, "null context");
    if (enable && !c->prof) c->prof = new EventProf();
    if (!enable && c->prof) {
        delete c->prof;
        c->prof = nullptr;
    }
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_profile_read(gs_ctx* c, gs_kernel_time* out, int max, int* n_out) try {
    clear_error();
    if (!c || !c->prof) return set_error(GS_ESTATE, "profiling is off");
    c->prof->collect();
    int n = 0;
    for (int k = 0; k < KT_COUNT; ++k) {
        if (!c->prof->launches[k]) continue;
        if (out && n < max) {
            std::memset(&out[n], 0, sizeof(gs_kernel_time));
            std::strncpy(out[n].name, kernel_name(k), sizeof(out[n].name) - 1);
            out[n].launches = c->prof->launches[k];
            out[n].total_ms = c->prof->total_ms[k];
        }
        ++n;
        c->prof->launches[k] = 0;
        c->prof->total_ms[k] = 0.0;
    }
    if (n_out) *n_out = n;
    return GS_OK;
} GS_ABI_CATCH

extern "C" void gs_destroy(gs_ctx* c) {
    if (!c) return;
    delete c->prof;
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
}

extern "C" size_t gs_ctx_bytes(const gs_ctx* c) { return c ? c->used.load() : (size_t)0; }

extern "C" gs_status gs_set_graphs(gs_ctx* c, int enable) try {
    if (!c) return set_error(GS_EINVAL, "null context");
    c->graphs = enable != 0;
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_mesh_set_act_seq(gs_mesh* m, const float* act, const float* hact, int n_steps, int mem,
                                         void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    if (n_steps < 0) return set_error(GS_EINVAL, "n_steps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t E = m->info.n_elems, B = m->info.n_hinges;
    if (mem == GS_MEM_HOST && n_steps > 0) {
        auto finite = [](const float* a, size_t n) {
            for (size_t i = 0; i < n; ++i)
                if (!std::isfinite(a[i])) return false;
            return true;
        };
        if ((act && !finite(act, (size_t)n_steps * E)) || (hact && !finite(hact, (size_t)n_steps * B)))
            return set_error(GS_EINVAL, "non-finite actuation sequence");
    }
    m->rt.act_seq = m->rt.hact_seq = nullptr;
    m->rt.n_act = 0;
    m->act_seq.release(s);
    m->hact_seq.release(s);
    if (n_steps == 0 || (!act && !hact)) return GS_OK;
    Buf tmp;
    const float* src = nullptr;
    if (act) {
        GS_TRY(stage_in(m->ctx, tmp, act, (size_t)n_steps * E, mem, s, &src));
        GS_TRY(m->act_seq.alloc(m->ctx, (size_t)n_steps * m->rt.act_ld * sizeof(float), s));
        launch_permute_rows(src, (float*)m->act_seq.p, n_steps, (int)E, m->rt.act_ld, (const int*)m->elem_perm.p, 1,
                            s);
        m->rt.act_seq = (const float*)m->act_seq.p;
    }
    if (hact && B > 0) {
        Buf tmp2;
        GS_TRY(stage_in(m->ctx, tmp2, hact, (size_t)n_steps * B, mem, s, &src));
        GS_TRY(m->hact_seq.alloc(m->ctx, (size_t)n_steps * m->rt.hact_ld * sizeof(float), s));
        launch_permute_rows(src, (float*)m->hact_seq.p, n_steps, (int)B, m->rt.hact_ld, (const int*)m->hinge_perm.p,
                            1, s);
        m->rt.hact_seq = (const float*)m->hact_seq.p;
        tmp2.release(s);
    }
    m->rt.n_act = n_steps;
    tmp.release(s);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_mesh_set_air(gs_mesh* m, const gs_air* air, void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    if (!air) {
        m->rt.air_on = 0;
        return GS_OK;
    }
    if (m->info.kind != GS_CLOTH) return set_error(GS_EINVAL, "the air model acts on cloth triangles (GS_CLOTH)");
    const float vals[5] = {air->k_drag, air->k_lift, air->wind[0], air->wind[1], air->wind[2]};
    for (float v : vals)
        if (!std::isfinite(v)) return set_error(GS_EINVAL, "non-finite air parameter");
    if (air->k_drag < 0.f || air->k_lift < 0.f) return set_error(GS_EINVAL, "air coefficients must be >= 0");
    // the adjoint's boundary partials of dL/dv: one per (boundary node, patch)
    if (!m->partials_v.p) GS_TRY(m->partials_v.alloc(m->ctx, m->partials.bytes, (cudaStream_t)stream));
    m->rt.partials_v = (float4*)m->partials_v.p;
    m->rt.k_drag = air->k_drag;
    m->rt.k_lift = air->k_lift;
    m->rt.wx = air->wind[0];
    m->rt.wy = air->wind[1];
    m->rt.wz = air->wind[2];
    m->rt.air_on = (air->k_drag > 0.f || air->k_lift > 0.f) ? 1 : 0;
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_step(gs_mesh* m, float dt, int n, void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    if (n < 0) return set_error(GS_EINVAL, "n_steps must be >= 0");
    return m->self->step(std::vector<float>{dt}, n, (cudaStream_t)stream);
} GS_ABI_CATCH

extern "C" gs_status gs_rollout(gs_mesh* m, float dt, int S, int K, const float* target, double* loss_out, int mem,
                                void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    cudaStream_t s = (cudaStream_t)stream;
    Buf tt;
    const float* dtarget = nullptr;
    GS_TRY(stage_in(m->ctx, tt, target, 3 * (size_t)m->info.n_nodes, mem, s, &dtarget));
    double* dloss = nullptr;
    Buf tl;
    if (loss_out) {
        if (mem == GS_MEM_DEVICE) dloss = loss_out;
        else {
            GS_TRY(tl.alloc(m->ctx, sizeof(double), s));
            dloss = (double*)tl.p;
        }
    }
    if (loss_out && !dtarget) return set_error(GS_EINVAL, "loss_out needs a target");
    gs_status st = m->self->rollout(std::vector<float>{dt}, S, K, std::vector<const float*>{dtarget}, dloss, s);
    if (st < 0) return st;
    if (loss_out && mem == GS_MEM_HOST) {
        GS_CUDA(cudaMemcpyAsync(loss_out, dloss, sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaStreamSynchronize(s));
    }
    tt.release(s);
    tl.release(s);
    return st;
} GS_ABI_CATCH

extern "C" gs_status gs_adjoint(gs_mesh* m, const float* dLdx, const float* dLdv, const gs_grads* grads, int mem,
                                int keep, void* stream) try {
    clear_error();
    if (!m) return set_error(GS_EINVAL, "null mesh");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n3 = 3 * (size_t)m->info.n_nodes;
    Buf t1, t2;
    const float *sx = nullptr, *sv = nullptr;
    GS_TRY(stage_in(m->ctx, t1, dLdx, n3, mem, s, &sx));
    GS_TRY(stage_in(m->ctx, t2, dLdv, n3, mem, s, &sv));
    gs_grads g{};
    if (grads) g = *grads;
    if (mem == GS_MEM_DEVICE) {
        GS_TRY(m->self->adjoint({sx}, {sv}, {g}, keep, s));
        return GS_OK;
    }
    // host gradients: compute into device scratch, then copy back
    const size_t E = m->info.n_elems, B = m->info.n_hinges, N = m->info.n_nodes;
    const size_t S = m->ro.valid ? (size_t)m->ro.S : 0;
    Buf hb;
    const size_t bytes = sizeof(double) * (4 * E + 2 * B + N) + sizeof(float) * 2 * n3 +
                         sizeof(float) * S * ((g.d_act_seq ? E : 0) + (g.d_hinge_act_seq ? B : 0));
    GS_TRY(hb.alloc(m->ctx, bytes, s));
    char* p = (char*)hb.p;
    gs_grads dg{};
    auto take = [&](size_t nbytes) {
        char* q = p;
        p += nbytes;
        return (void*)q;
    };
    dg.d_mu = g.d_mu ? (double*)take(8 * E) : nullptr;
    dg.d_lambda = g.d_lambda ? (double*)take(8 * E) : nullptr;
    dg.d_density = g.d_density ? (double*)take(8 * E) : nullptr;
    dg.d_act = g.d_act ? (double*)take(8 * E) : nullptr;
    dg.d_kb = g.d_kb ? (double*)take(8 * B) : nullptr;
    dg.d_hinge_act = g.d_hinge_act ? (double*)take(8 * B) : nullptr;
    dg.d_mass = g.d_mass ? (double*)take(8 * N) : nullptr;
    dg.d_x0 = g.d_x0 ? (float*)take(4 * n3) : nullptr;
    dg.d_v0 = g.d_v0 ? (float*)take(4 * n3) : nullptr;
    dg.d_act_seq = g.d_act_seq ? (float*)take(4 * S * E) : nullptr;
    dg.d_hinge_act_seq = g.d_hinge_act_seq ? (float*)take(4 * S * B) : nullptr;
    GS_TRY(m->self->adjoint({sx}, {sv}, {dg}, keep, s));
    auto back = [&](void* dst, const void* src, size_t nbytes) -> gs_status {
        if (dst && src) GS_CUDA(cudaMemcpyAsync(dst, src, nbytes, cudaMemcpyDeviceToHost, s));
        return GS_OK;
    };
    GS_TRY(back(g.d_mu, dg.d_mu, 8 * E));
    GS_TRY(back(g.d_lambda, dg.d_lambda, 8 * E));
    GS_TRY(back(g.d_density, dg.d_density, 8 * E));
    GS_TRY(back(g.d_act, dg.d_act, 8 * E));
    GS_TRY(back(g.d_kb, dg.d_kb, 8 * B));
    GS_TRY(back(g.d_hinge_act, dg.d_hinge_act, 8 * B));
    GS_TRY(back(g.d_mass, dg.d_mass, 8 * N));
    GS_TRY(back(g.d_x0, dg.d_x0, 4 * n3));
    GS_TRY(back(g.d_v0, dg.d_v0, 4 * n3));
    GS_TRY(back(g.d_act_seq, dg.d_act_seq, 4 * S * E));
    GS_TRY(back(g.d_hinge_act_seq, dg.d_hinge_act_seq, 4 * S * B));
    GS_CUDA(cudaStreamSynchronize(s));
    hb.release(s);
    t1.release(s);
    t2.release(s);
    return GS_OK;
} GS_ABI_CATCH

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct gs_batch {
    gs_ctx* ctx = nullptr;
    std::vector<gs_mesh*> meshes;
    std::unique_ptr<LaunchSet> ls;
};

extern "C" gs_status gs_batch_create(gs_ctx* ctx, gs_mesh* const* meshes, int n, gs_batch** out) try {
    clear_error();
    if (!ctx || !meshes || n <= 0 || !out) return set_error(GS_EINVAL, "bad batch arguments");
    *out = nullptr;
    std::unique_ptr<gs_batch> b(new gs_batch());
    b->ctx = ctx;
    b->meshes.assign(meshes, meshes + n);
    for (gs_mesh* m : b->meshes)
        if (!m || m->ctx != ctx) return set_error(GS_EINVAL, "batch meshes must belong to the context");
    b->ls.reset(new LaunchSet());
    GS_TRY(b->ls->build(ctx, b->meshes, 0));
    GS_CUDA(cudaStreamSynchronize(0));
    *out = b.release();
    return GS_OK;
} GS_ABI_CATCH

extern "C" void gs_batch_destroy(gs_batch* b) { delete b; }

extern "C" gs_status gs_batch_step(gs_batch* b, const float* dt, int n, void* stream) try {
    clear_error();
    if (!b || !dt) return set_error(GS_EINVAL, "null argument");
    return b->ls->step(std::vector<float>(dt, dt + b->meshes.size()), n, (cudaStream_t)stream);
} GS_ABI_CATCH

extern "C" gs_status gs_batch_rollout(gs_batch* b, const float* dt, int S, int K, const float* const* targets,
                                      double* loss_out, void* stream) try {
    clear_error();
    if (!b || !dt) return set_error(GS_EINVAL, "null argument");
    std::vector<const float*> t(b->meshes.size(), nullptr);
    if (targets)
        for (size_t i = 0; i < t.size(); ++i) t[i] = targets[i];
    return b->ls->rollout(std::vector<float>(dt, dt + b->meshes.size()), S, K, t, loss_out, (cudaStream_t)stream);
} GS_ABI_CATCH

extern "C" gs_status gs_batch_adjoint(gs_batch* b, const gs_grads* grads, void* stream) try {
    clear_error();
    if (!b) return set_error(GS_EINVAL, "null argument");
    const size_t n = b->meshes.size();
    std::vector<const float*> z(n, nullptr);
    std::vector<gs_grads> g(n, gs_grads{});
    if (grads)
        for (size_t i = 0; i < n; ++i) g[i] = grads[i];
    return b->ls->adjoint(z, z, g, 0, (cudaStream_t)stream);
} GS_ABI_CATCH
