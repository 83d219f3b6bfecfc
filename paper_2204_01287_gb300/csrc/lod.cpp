// lod.cpp — layered-octree level of detail (Sec. 3.5): host builder
// (pc_lod_encode) and pc_build_lod, which decodes a resident cloud at full
// precision, builds the tree and uploads it as a LOD cloud.
//
// Tree: the root is the cubic box of the cloud (corner = per-axis minimum,
// side = largest extent). A node with more than max_node_points points and a
// depth below max_levels - 1 keeps the max_node_points points of smallest
// priority SplitMix64(seed * 2^32 + index) (ties by index), a uniform subset,
// and passes the rest to its octant children (upper half when p >= corner +
// side/2); other nodes keep all their points. The tree is additive: every
// point lives in exactly one node. Nodes are numbered breadth first, children
// in octant order (bit 0 x, bit 1 y, bit 2 z); each node's points keep the
// input order and are quantized with Eq. 1 against the node's cube.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "pc_api_internal.h"

namespace pcr {

namespace {

inline uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class F>
void run_threads(unsigned threads, F&& f) {
    if (threads <= 1) {
        f(0u);
        return;
    }
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < threads; ++t) pool.emplace_back(f, t);
    for (auto& th : pool) th.join();
}

// Eq. 1 in binary64 from binary32 inputs (the same formula as the encoder).
inline uint32_t fixed30(float v, float bmin, float bsize) {
    if (!(bsize > 0.0f)) return 0;
    double t = std::floor(1073741824.0 * ((double)v - (double)bmin) / (double)bsize);
    t = t < 0.0 ? 0.0 : (t > 1073741823.0 ? 1073741823.0 : t);
    return (uint32_t)t;
}

struct Item {
    float lo[3];
    float size;
    uint32_t level;
    uint32_t parent;
    std::vector<uint32_t> idx;        // points of the node and its subtree, input order
    std::vector<uint32_t> kept;       // the node's own points, input order
    std::vector<uint32_t> rest[8];    // the children's points per octant, input order
};

struct Pri {
    uint64_t p;
    uint32_t i;
    bool operator<(const Pri& o) const { return p != o.p ? p < o.p : i < o.i; }
};

// Split one item into kept points and octant groups, using `threads` threads.
void process_item(Item& it, uint32_t max_levels, uint32_t M, uint32_t seed, unsigned threads,
                  const float* xyz) {
    const uint64_t n = it.idx.size();
    if (n <= M || it.level + 1 >= max_levels) {
        it.kept.swap(it.idx);
        return;
    }
    // the M smallest (priority, index): filter candidates under a threshold
    // that keeps about 1.25 M of them in expectation, then select exactly
    const uint64_t base = (uint64_t)seed << 32;
    double frac = std::min(1.0, 1.25 * (double)M / (double)n + 64.0 / (double)n);
    Pri cut{0, 0};
    for (;;) {
        const uint64_t t = frac >= 1.0 ? ~0ull : (uint64_t)(frac * 18446744073709551615.0);
        std::vector<std::vector<Pri>> cand(threads);
        run_threads(threads, [&](unsigned th) {
            const uint64_t lo = n * th / threads, hi = n * (th + 1) / threads;
            for (uint64_t j = lo; j < hi; ++j) {
                const uint32_t i = it.idx[j];
                const uint64_t p = splitmix64(base + i);
                if (p <= t) cand[th].push_back({p, i});
            }
        });
        std::vector<Pri> all;
        for (auto& c : cand) all.insert(all.end(), c.begin(), c.end());
        if (all.size() >= M) {
            std::nth_element(all.begin(), all.begin() + (M - 1), all.end());
            cut = all[M - 1];
            break;
        }
        frac = std::min(1.0, frac * 2.0);
    }
    // stable split: kept (priority <= cut) and octant groups of the rest
    const float half = it.size * 0.5f;
    float mid[3];
    for (int a = 0; a < 3; ++a) mid[a] = it.lo[a] + half;
    std::vector<std::vector<uint32_t>> k_parts(threads);
    std::vector<std::vector<uint32_t>> r_parts(threads * 8);
    run_threads(threads, [&](unsigned th) {
        const uint64_t lo = n * th / threads, hi = n * (th + 1) / threads;
        for (uint64_t j = lo; j < hi; ++j) {
            const uint32_t i = it.idx[j];
            const Pri pr{splitmix64(base + i), i};
            if (!(cut < pr)) {
                k_parts[th].push_back(i);
            } else {
                const float* p = &xyz[3 * (uint64_t)i];
                const int o = (p[0] >= mid[0]) | ((p[1] >= mid[1]) << 1) | ((p[2] >= mid[2]) << 2);
                r_parts[th * 8 + o].push_back(i);
            }
        }
    });
    for (auto& k : k_parts) it.kept.insert(it.kept.end(), k.begin(), k.end());
    for (int o = 0; o < 8; ++o)
        for (unsigned th = 0; th < threads; ++th)
            it.rest[o].insert(it.rest[o].end(), r_parts[th * 8 + o].begin(),
                              r_parts[th * 8 + o].end());
    std::vector<uint32_t>().swap(it.idx);
}

}  // namespace

pc_status lod_encode_host(const float* xyz, const uint32_t* rgba, uint64_t n,
                          uint32_t max_levels, uint32_t M, uint32_t seed, unsigned threads,
                          std::vector<pc_batch>& nodes, std::vector<uint32_t>& parent,
                          std::vector<uint32_t>& level, uint32_t* perm, uint32_t* w1,
                          uint32_t* w2, uint32_t* w3, uint32_t* color) {
    nodes.clear();
    parent.clear();
    level.clear();
    if (n == 0) return PC_OK;
    if (n >= 0xFFFFFFFFull || max_levels == 0 || M == 0) return PC_EINVAL;
    if (threads == 0) threads = hw_threads();
    if (!coords_finite(xyz, n, threads)) return PC_EINVAL;   // the root cube must be finite
    // root cube
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = xyz[a];
    for (uint64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            const float v = xyz[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    float side = 0.0f;
    for (int a = 0; a < 3; ++a) {
        const float e = hi[a] - lo[a];
        if (e > side) side = e;
    }
    std::vector<std::unique_ptr<Item>> cur;
    {
        auto root = std::make_unique<Item>();
        for (int a = 0; a < 3; ++a) root->lo[a] = lo[a];
        root->size = side;
        root->level = 0;
        root->parent = 0;
        root->idx.resize(n);
        for (uint64_t i = 0; i < n; ++i) root->idx[i] = (uint32_t)i;
        cur.push_back(std::move(root));
    }
    uint64_t out = 0;
    while (!cur.empty()) {
        // split the level's items: big ones with all threads, the others in parallel
        std::atomic<size_t> next{0};
        for (auto& it : cur)
            if (it->idx.size() > (1u << 22)) process_item(*it, max_levels, M, seed, threads, xyz);
        run_threads(threads, [&](unsigned) {
            for (;;) {
                const size_t k = next.fetch_add(1);
                if (k >= cur.size()) break;
                Item& it = *cur[k];
                if (!it.idx.empty() && it.kept.empty())
                    process_item(it, max_levels, M, seed, 1, xyz);
            }
        });
        // number the level's nodes, place their points, queue the children
        const uint32_t id0 = (uint32_t)nodes.size();
        std::vector<uint64_t> first(cur.size());
        std::vector<std::unique_ptr<Item>> nxt;
        for (size_t k = 0; k < cur.size(); ++k) {
            Item& it = *cur[k];
            pc_batch b;
            for (int a = 0; a < 3; ++a) {
                b.min[a] = it.lo[a];
                b.size[a] = it.size;
            }
            b.first = (uint32_t)out;
            b.count = (uint32_t)it.kept.size();
            first[k] = out;
            out += it.kept.size();
            nodes.push_back(b);
            parent.push_back(it.parent);
            level.push_back(it.level);
            const float half = it.size * 0.5f;
            for (int o = 0; o < 8; ++o) {
                if (it.rest[o].empty()) continue;
                auto c = std::make_unique<Item>();
                for (int a = 0; a < 3; ++a) c->lo[a] = ((o >> a) & 1) ? it.lo[a] + half : it.lo[a];
                c->size = half;
                c->level = it.level + 1;
                c->parent = id0 + (uint32_t)k;
                c->idx.swap(it.rest[o]);
                nxt.push_back(std::move(c));
            }
        }
        // Eq. 1 against each node's cube
        next = 0;
        run_threads(threads, [&](unsigned) {
            for (;;) {
                const size_t k = next.fetch_add(1);
                if (k >= cur.size()) break;
                const Item& it = *cur[k];
                const pc_batch& b = nodes[id0 + k];
                for (size_t j = 0; j < it.kept.size(); ++j) {
                    const uint32_t i = it.kept[j];
                    const float* p = &xyz[3 * (uint64_t)i];
                    const uint32_t q0 = fixed30(p[0], b.min[0], b.size[0]);
                    const uint32_t q1 = fixed30(p[1], b.min[1], b.size[1]);
                    const uint32_t q2 = fixed30(p[2], b.min[2], b.size[2]);
                    const uint64_t o = first[k] + j;
                    perm[o] = i;
                    w1[o] = (q0 >> 20) | ((q1 >> 20) << 10) | ((q2 >> 20) << 20);
                    w2[o] = ((q0 >> 10) & 1023u) | (((q1 >> 10) & 1023u) << 10) |
                            (((q2 >> 10) & 1023u) << 20);
                    w3[o] = (q0 & 1023u) | ((q1 & 1023u) << 10) | ((q2 & 1023u) << 20);
                    color[o] = rgba ? rgba[i] : 0u;
                }
            }
        });
        cur.swap(nxt);
    }
    return PC_OK;
}

}  // namespace pcr

using namespace pcr;

extern "C" pc_status pc_lod_encode(const float* xyz, const uint32_t* rgba, uint64_t n,
                                   const pc_lod_opts* opts, uint32_t threads,
                                   uint64_t max_nodes, pc_batch* nodes, uint32_t* parent,
                                   uint32_t* level, uint64_t* n_nodes, uint32_t* perm,
                                   uint32_t* w1, uint32_t* w2, uint32_t* w3, uint32_t* color) {
    if (!n_nodes || (n && (!xyz || !perm || !w1 || !w2 || !w3 || !color))) return PC_EINVAL;
    pc_lod_opts o{12, 10240, 0, 0};
    if (opts) o = *opts;
    if (o.max_levels == 0 || o.max_node_points == 0) return PC_EINVAL;
    std::vector<pc_batch> nb;
    std::vector<uint32_t> par, lev;
    pc_status rc;
    try {
        rc = lod_encode_host(xyz, rgba, n, o.max_levels, o.max_node_points, o.seed, threads, nb,
                             par, lev, perm, w1, w2, w3, color);
    } catch (...) {
        return PC_ENOMEM;
    }
    if (rc != PC_OK) return rc;
    *n_nodes = nb.size();
    if (nb.size() > max_nodes) return PC_ENOMEM;
    if (nb.size() && (!nodes || !parent || !level)) return PC_EINVAL;
    std::memcpy(nodes, nb.data(), nb.size() * sizeof(pc_batch));
    std::memcpy(parent, par.data(), par.size() * sizeof(uint32_t));
    std::memcpy(level, lev.data(), lev.size() * sizeof(uint32_t));
    return PC_OK;
}

static pc_status build_lod(pc_ctx* h, Ctx& ctx, pc_cloud src, const pc_lod_opts& o,
                           pc_cloud* out) {
    auto cl = ctx.find_cloud(src);
    if (!cl) return PC_ENOTFOUND;
    if (cl->is_lod) {
        ctx.fail_msg("pc_build_lod: the source is already a LOD cloud");
        return PC_ENOTSUP;
    }
    cudaSetDevice(ctx.device);
    const uint64_t n = cl->n_points, nb = cl->n_batches;
    std::vector<pc_batch> batches(nb);
    std::vector<uint32_t> w1(n), w2(n), w3(n), col(n);
    pc_status rc = pc_cloud_download(h, src, batches.data(), w1.data(), w2.data(), w3.data(),
                                     col.data());
    if (rc != PC_OK) return rc;
    // full-precision decoded positions (Sec. 3.3, k = 3): min + float(X30) * size * 2^-30
    std::vector<float> xyz(3 * n);
    const unsigned threads = ctx.cfg.encoder_threads ? ctx.cfg.encoder_threads : hw_threads();
    std::atomic<uint64_t> next{0};
    run_threads(threads, [&](unsigned) {
        for (;;) {
            const uint64_t b = next.fetch_add(1);
            if (b >= nb) break;
            const pc_batch& B = batches[b];
            float cell[3];
            for (int a = 0; a < 3; ++a) cell[a] = std::ldexp(B.size[a], -30);
            for (uint32_t j = 0; j < B.count; ++j) {
                const uint64_t i = (uint64_t)B.first + j;
                for (int a = 0; a < 3; ++a) {
                    const uint32_t q = (((w1[i] >> (10 * a)) & 1023u) << 20) |
                                       (((w2[i] >> (10 * a)) & 1023u) << 10) |
                                       ((w3[i] >> (10 * a)) & 1023u);
                    const float off = (float)q * cell[a];
                    xyz[3 * i + a] = B.min[a] + off;
                }
            }
        }
    });
    std::vector<pc_batch> nodes;
    std::vector<uint32_t> parent, level, perm(n), l1(n), l2(n), l3(n), lc(n);
    try {
        rc = lod_encode_host(xyz.data(), col.data(), n, o.max_levels, o.max_node_points, o.seed,
                             threads, nodes, parent, level, perm.data(), l1.data(), l2.data(),
                             l3.data(), lc.data());
    } catch (...) {
        rc = PC_ENOMEM;
    }
    if (rc != PC_OK) return rc;
    std::shared_ptr<Cloud> lod;
    rc = upload_encoded_internal(ctx, nodes.data(), nodes.size(), l1.data(), l2.data(),
                                 l3.data(), lc.data(), n, lod);
    if (rc != PC_OK) return rc;
    const size_t nn = std::max<size_t>(1, nodes.size());
    cudaError_t e = cudaMalloc(&lod->parent, nn * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&lod->level, nn * sizeof(uint32_t));
    if (e == cudaSuccess && !nodes.empty())
        e = cudaMemcpy(lod->parent, parent.data(), nodes.size() * sizeof(uint32_t),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !nodes.empty())
        e = cudaMemcpy(lod->level, level.data(), nodes.size() * sizeof(uint32_t),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return ctx.cuda_fail(e, "LOD hierarchy upload");
    lod->is_lod = 1;
    uint32_t maxl = 0;
    for (uint32_t l : level) maxl = std::max(maxl, l);
    lod->lod_levels = nodes.empty() ? 0 : maxl + 1;
    lod->device_bytes += 2 * nn * sizeof(uint32_t);
    *out = ctx.register_cloud(lod);
    return PC_OK;
}

extern "C" pc_status pc_build_lod(pc_ctx* h, pc_cloud src, const pc_lod_opts* opts,
                                  pc_cloud* out) {
    if (!h || !out) return PC_EINVAL;
    Ctx& ctx = *reinterpret_cast<Ctx*>(h);
    *out = 0;
    pc_lod_opts o{12, 10240, 0, 0};
    if (opts) o = *opts;
    if (o.max_levels == 0 || o.max_node_points == 0) return PC_EINVAL;
    try {   // the host copies of the cloud and the tree are a few times its size
        return build_lod(h, ctx, src, o, out);
    } catch (const std::exception& e) {
        ctx.fail_msg("pc_build_lod: %s", e.what());
        return PC_ENOMEM;
    }
}
