// emd_topk_merge: the exact global top-K of a database split into document shards (one
// per process or device), from each shard's own top-K.  Every document of the global top-K
// is in its shard's top-K, so the K smallest (distance, global id) pairs of the union are
// the global answer.  Host code only: it needs no device.

#include <algorithm>
#include <cstdint>
#include <vector>

#include "emd.h"
#include "emd_db.cuh"

emd_status emd_topk_merge(int32_t n_shards, const int64_t* const* shard_idx, const float* const* shard_dist,
                          const int64_t* id_offset, int64_t n_queries, int32_t K_shard, int32_t K,
                          int64_t* out_idx, float* out_dist)
{
    emd::clear_error();
    if (n_shards < 1 || !shard_idx || !shard_dist || !id_offset || !out_idx || !out_dist)
        return emd::fail(EMD_ERR_INVALID_ARG, "NULL argument or no shard");
    if (n_queries < 0 || K < 1 || K_shard < 1 || (int64_t)K > (int64_t)n_shards * K_shard)
        return emd::fail(EMD_ERR_INVALID_ARG, "need 1 <= K <= n_shards * K_shard");
    for (int32_t s = 0; s < n_shards; ++s)
        if (!shard_idx[s] || !shard_dist[s]) return emd::fail(EMD_ERR_INVALID_ARG, "shard %d is NULL", s);
    struct Key {
        float d;
        int64_t id;
    };
    std::vector<Key> all((size_t)n_shards * K_shard);
    for (int64_t q = 0; q < n_queries; ++q) {
        size_t c = 0;
        for (int32_t s = 0; s < n_shards; ++s)
            for (int32_t l = 0; l < K_shard; ++l) {
                const int64_t local = shard_idx[s][q * K_shard + l];
                if (local < 0) continue;  // a shard with fewer than K_shard documents
                all[c++] = {shard_dist[s][q * K_shard + l], local + id_offset[s]};
            }
        if ((int64_t)c < K) return emd::fail(EMD_ERR_INVALID_ARG, "query %lld: fewer than K results", (long long)q);
        std::partial_sort(all.begin(), all.begin() + K, all.begin() + c, [](const Key& a, const Key& b) {
            return a.d < b.d || (a.d == b.d && a.id < b.id);
        });
        for (int32_t l = 0; l < K; ++l) {
            out_idx[q * K + l] = all[l].id;
            out_dist[q * K + l] = all[l].d;
        }
    }
    return EMD_OK;
}
