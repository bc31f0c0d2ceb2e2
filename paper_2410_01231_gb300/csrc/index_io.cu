// index_io.cu -- writing an index to a file and reading it back.
//
// The layout (little-endian, version 1) is stated in pg.h beside
// pg_index_save.  Reading checks the whole file on the host before the
// index is handed out, so that a damaged or foreign file can never put an
// out-of-range id in front of a kernel: layer 0 holds every point, an upper
// layer holds strictly ascending ids that are members of the layer below,
// every listed neighbour is a member of its own layer, degrees are within
// [0, R], the entry points exist, and a checksum over the whole file
// matches.  Only plain copies touch the device.
#include <algorithm>
#include <cerrno>
#include <climits>
#include <cstdarg>
#include <cstring>
#include <functional>

#include "pg_internal.cuh"

namespace {

constexpr char kMagic[8] = {'P', 'G', 'I', 'N', 'D', 'E', 'X', '\0'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kByteOrder = 0x01020304u;
constexpr int kMaxLayers = 64;
constexpr size_t kChunk = size_t(16) << 20;  // bytes per staged copy of the points

// FNV-1a over little-endian 64-bit words (last partial word zero-padded).
struct Fnv64 {
    uint64_t h = 0xcbf29ce484222325ULL;
    uint8_t carry[8] = {0};
    int nc = 0;
    static uint64_t le64(const uint8_t *b) {
        uint64_t w = 0;
        for (int i = 7; i >= 0; --i) w = (w << 8) | b[i];
        return w;
    }
    void word(uint64_t w) {
        h ^= w;
        h *= 0x100000001b3ULL;
    }
    void add(const void *p, size_t len) {
        const uint8_t *b = static_cast<const uint8_t *>(p);
        while (len && nc) {
            carry[nc++] = *b++;
            --len;
            if (nc == 8) {
                word(le64(carry));
                nc = 0;
            }
        }
        for (; len >= 8; b += 8, len -= 8) word(le64(b));
        while (len) {
            carry[nc++] = *b++;
            --len;
        }
    }
    uint64_t finish() {
        if (nc) {
            std::fill(carry + nc, carry + 8, uint8_t(0));
            word(le64(carry));
            nc = 0;
        }
        return h;
    }
};

struct FileHeader {
    int64_t n = 0;
    int32_t d = 0, metric = 0;
    int64_t ep_top = 0, ep_base = 0;
    pg_build_params p{};
    int32_t layers = 0;
    int64_t count[kMaxLayers] = {0};
    int32_t R[kMaxLayers] = {0};
    int32_t has_gid[kMaxLayers] = {0};
};

// ------------------------------------------------------------------ writing

struct Writer {
    FILE *f = nullptr;
    Fnv64 hash;
    bool ok = true;
    void put(const void *p, size_t len) {
        if (!ok || !len) return;
        hash.add(p, len);
        ok = fwrite(p, 1, len, f) == len;
    }
    template <class T>
    void val(T v) {
        put(&v, sizeof v);
    }
};

void write_header(Writer &w, const FileHeader &h) {
    w.put(kMagic, 8);
    w.val<uint32_t>(kVersion);
    w.val<uint32_t>(kByteOrder);
    w.val<int64_t>(h.n);
    w.val<int32_t>(h.d);
    w.val<int32_t>(h.metric);
    w.val<int64_t>(h.ep_top);
    w.val<int64_t>(h.ep_base);
    w.val<int32_t>((int32_t)h.p.metric);
    w.val<int32_t>((int32_t)h.p.precision);
    w.val<int32_t>(h.p.K);
    w.val<int32_t>(h.p.L);
    w.val<int32_t>(h.p.R);
    w.val<int32_t>(h.p.M);
    w.val<double>(h.p.alpha_deg);
    w.val<double>(h.p.alpha_final_deg);
    w.val<int32_t>(h.p.iters);
    w.val<int32_t>(h.p.connect_final);
    w.val<int32_t>(h.p.route_layers);
    w.val<int32_t>(0);
    w.val<uint64_t>(h.p.seed);
    w.val<int32_t>(h.layers);
    w.val<int32_t>(0);
    for (int i = 0; i < h.layers; ++i) {
        w.val<int64_t>(h.count[i]);
        w.val<int32_t>(h.R[i]);
        w.val<int32_t>(h.has_gid[i]);
    }
}

// ------------------------------------------------------------------ reading

struct Reader {
    FILE *f = nullptr;
    Fnv64 hash;
    pg_status st = PG_OK;
    std::string msg;
    bool fail(pg_status s, const char *fmt, ...) {
        if (st != PG_OK) return false;
        char buf[256];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        st = s;
        msg = buf;
        return false;
    }
    bool get(void *p, size_t len, const char *what) {
        if (st != PG_OK) return false;
        if (len && fread(p, 1, len, f) != len)
            return fail(PG_ERR_IO, "index file: short read in %s", what);
        hash.add(p, len);
        return true;
    }
    template <class T>
    bool val(T *v, const char *what) {
        return get(v, sizeof *v, what);
    }
};

bool read_header(Reader &r, FileHeader &h) {
    char magic[8];
    uint32_t version = 0, bom = 0;
    if (!r.get(magic, 8, "magic")) return false;
    if (memcmp(magic, kMagic, 8) != 0) return r.fail(PG_ERR_INVALID_ARG, "not an index file");
    if (!r.val(&version, "version") || !r.val(&bom, "byte order")) return false;
    if (bom != kByteOrder) return r.fail(PG_ERR_INVALID_ARG, "index file: foreign byte order");
    if (version != kVersion)
        return r.fail(PG_ERR_INVALID_ARG, "index file: version %u, expected %u", version, kVersion);
    int32_t pm = 0, pp = 0, pad = 0;
    bool ok = r.val(&h.n, "n") && r.val(&h.d, "d") && r.val(&h.metric, "metric") &&
              r.val(&h.ep_top, "ep_top") && r.val(&h.ep_base, "ep_base") &&
              r.val(&pm, "params") && r.val(&pp, "params") && r.val(&h.p.K, "params") &&
              r.val(&h.p.L, "params") && r.val(&h.p.R, "params") && r.val(&h.p.M, "params") &&
              r.val(&h.p.alpha_deg, "params") && r.val(&h.p.alpha_final_deg, "params") &&
              r.val(&h.p.iters, "params") && r.val(&h.p.connect_final, "params") &&
              r.val(&h.p.route_layers, "params") && r.val(&pad, "params") &&
              r.val(&h.p.seed, "params") && r.val(&h.layers, "layers") && r.val(&pad, "layers");
    if (!ok) return false;
    h.p.metric = (pg_metric)pm;
    h.p.precision = (pg_precision)pp;
    // the ranges the builds accept
    if (h.n < 2 || h.n >= INT_MAX) return r.fail(PG_ERR_INVALID_ARG, "index file: bad n");
    if (h.d < 4 || h.d % 4 || h.d > 8192) return r.fail(PG_ERR_INVALID_ARG, "index file: bad d");
    if (h.metric < PG_METRIC_L2SQ || h.metric > PG_METRIC_IP || pm != h.metric)
        return r.fail(PG_ERR_INVALID_ARG, "index file: bad metric");
    if (pp < PG_PREC_FP32 || pp > PG_PREC_BF16_SCREEN)
        return r.fail(PG_ERR_INVALID_ARG, "index file: bad precision");
    const pg_build_params &p = h.p;
    if (p.K < 1 || p.K > 256 || p.L < 1 || p.L > 256 || p.R < 1 || p.R > 64 || p.M < 2 ||
        p.M > 64 || p.iters < 0 || p.iters > 16 ||
        !(p.alpha_deg >= 0 && p.alpha_deg <= 180 && p.alpha_final_deg >= 0 &&
          p.alpha_final_deg <= 180))
        return r.fail(PG_ERR_INVALID_ARG, "index file: build parameters out of range");
    if (h.layers < 1 || h.layers > kMaxLayers)
        return r.fail(PG_ERR_INVALID_ARG, "index file: bad layer count");
    if (h.ep_base < 0 || h.ep_base >= h.n || h.ep_top < 0 || h.ep_top >= h.n)
        return r.fail(PG_ERR_INVALID_ARG, "index file: entry point out of range");
    for (int i = 0; i < h.layers; ++i) {
        if (!r.val(&h.count[i], "layer table") || !r.val(&h.R[i], "layer table") ||
            !r.val(&h.has_gid[i], "layer table"))
            return false;
        const bool ok_layer =
            i == 0 ? (h.count[0] == h.n && h.has_gid[0] == 0 && h.R[0] == p.R)
                   : (h.count[i] >= 1 && h.count[i] <= h.count[i - 1] && h.has_gid[i] == 1 &&
                      h.R[i] == p.M);
        if (!ok_layer) return r.fail(PG_ERR_INVALID_ARG, "index file: bad shape of layer %d", i);
    }
    return true;
}

struct LayerHost {
    std::vector<int32_t> gid, deg, nbr;
};

// Read layer i into L and check it; `member` holds the members of layer
// i - 1 on entry (all points for i = 0) and of layer i on return.
bool read_layer(Reader &r, const FileHeader &h, int i, LayerHost &L,
                std::vector<uint8_t> &member) {
    const int64_t m = h.count[i], R = h.R[i], n = h.n;
    L.gid.clear();
    if (h.has_gid[i]) {
        L.gid.resize((size_t)m);
        if (!r.get(L.gid.data(), (size_t)m * 4, "layer members")) return false;
        std::vector<uint8_t> next((size_t)n, 0);
        for (int64_t t = 0; t < m; ++t) {
            const int32_t g = L.gid[(size_t)t];
            if (g < 0 || g >= n || (t && g <= L.gid[(size_t)t - 1]))
                return r.fail(PG_ERR_INVALID_ARG, "index file: layer %d members not ascending ids",
                              i);
            if (!member[(size_t)g])
                return r.fail(PG_ERR_INVALID_ARG,
                              "index file: layer %d member %d missing from the layer below", i, g);
            next[(size_t)g] = 1;
        }
        member.swap(next);
    }
    L.deg.resize((size_t)m);
    L.nbr.resize((size_t)(m * R));
    if (!r.get(L.deg.data(), (size_t)m * 4, "degrees")) return false;
    if (!r.get(L.nbr.data(), (size_t)(m * R) * 4, "neighbour lists")) return false;
    for (int64_t t = 0; t < m; ++t) {
        const int32_t dg = L.deg[(size_t)t];
        if (dg < 0 || dg > R)
            return r.fail(PG_ERR_INVALID_ARG, "index file: layer %d row %lld degree %d", i,
                          (long long)t, dg);
        for (int32_t j = 0; j < dg; ++j) {
            const int32_t v = L.nbr[(size_t)(t * R + j)];
            if (v < 0 || v >= n || !member[(size_t)v])
                return r.fail(PG_ERR_INVALID_ARG,
                              "index file: layer %d row %lld lists %d, not a member", i,
                              (long long)t, v);
        }
    }
    if (i == h.layers - 1 && !member[(size_t)h.ep_top])
        return r.fail(PG_ERR_INVALID_ARG, "index file: top entry point not in the top layer");
    return true;
}

// Parse a whole file; on_layer / on_points receive the checked contents
// (either may be empty: a check without a device).
pg_status parse_file_unguarded(const char *path, FileHeader &h, std::string &msg,
                               const std::function<bool(int, LayerHost &)> &on_layer,
                               const std::function<bool(const float *, int64_t, int64_t)> &on_points) {
    Reader r;
    r.f = fopen(path, "rb");
    if (!r.f) {
        msg = std::string("index file: cannot open: ") + strerror(errno);
        return PG_ERR_IO;
    }
    std::vector<uint8_t> member;
    LayerHost L;
    bool ok = read_header(r, h);
    if (ok) {
        // the size the header implies must be the file's size: nothing is
        // allocated for a truncated file or an inflated header
        int64_t expect = (int64_t)ftello(r.f) + (int64_t)h.n * h.d * 4 + 8;
        for (int i = 0; i < h.layers; ++i)
            expect += h.count[i] * 4 * ((h.has_gid[i] ? 2 : 1) + (int64_t)h.R[i]);
        const int64_t here = (int64_t)ftello(r.f);
        if (fseeko(r.f, 0, SEEK_END) != 0) {
            ok = r.fail(PG_ERR_IO, "index file: cannot seek");
        } else {
            const int64_t size = (int64_t)ftello(r.f);
            if (fseeko(r.f, (off_t)here, SEEK_SET) != 0)
                ok = r.fail(PG_ERR_IO, "index file: cannot seek");
            else if (size != expect)
                ok = r.fail(size < expect ? PG_ERR_IO : PG_ERR_INVALID_ARG,
                            "index file: %lld bytes, its header implies %lld", (long long)size,
                            (long long)expect);
        }
    }
    if (ok) member.assign((size_t)h.n, 1);
    for (int i = 0; ok && i < h.layers; ++i) {
        ok = read_layer(r, h, i, L, member);
        if (ok && on_layer && !on_layer(i, L)) ok = r.fail(PG_ERR_CUDA, "%s", "upload");
    }
    if (ok) {
        const int64_t per = std::max<int64_t>(1, (int64_t)(kChunk / ((size_t)h.d * 4)));
        std::vector<float> buf((size_t)(std::min(per, h.n) * h.d));
        for (int64_t r0 = 0; ok && r0 < h.n; r0 += per) {
            const int64_t rows = std::min(per, h.n - r0);
            ok = r.get(buf.data(), (size_t)(rows * h.d) * 4, "points");
            if (ok && on_points && !on_points(buf.data(), r0, rows))
                ok = r.fail(PG_ERR_CUDA, "%s", "upload");
        }
    }
    if (ok) {
        const uint64_t want = r.hash.finish();
        uint64_t got = 0;
        // the checksum itself is not hashed
        if (fread(&got, 1, 8, r.f) != 8)
            ok = r.fail(PG_ERR_IO, "index file: short read in checksum");
        else if (got != want)
            ok = r.fail(PG_ERR_INVALID_ARG, "index file: checksum mismatch");
        else if (fgetc(r.f) != EOF)
            ok = r.fail(PG_ERR_INVALID_ARG, "index file: trailing bytes after the checksum");
    }
    fclose(r.f);
    if (!ok) msg = r.msg;
    return ok ? PG_OK : r.st;
}

pg_status parse_file(const char *path, FileHeader &h, std::string &msg,
                     const std::function<bool(int, LayerHost &)> &on_layer,
                     const std::function<bool(const float *, int64_t, int64_t)> &on_points) {
    try {
        return parse_file_unguarded(path, h, msg, on_layer, on_points);
    } catch (const std::bad_alloc &) {
        msg = "index file: host allocation failed";
        return PG_ERR_OOM;
    }
}

template <class T>
pg_status upload(pg_ctx *ctx, T *&dst, const std::vector<T> &src) {
    PG_TRY_CUDA(ctx, cudaMalloc(&dst, std::max<size_t>(src.size(), 1) * sizeof(T)));
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T),
                                     cudaMemcpyHostToDevice, ctx->stream));
    return PG_OK;
}

}  // namespace

extern "C" pg_status pg_index_params(const pg_index *idx, pg_build_params *params, int32_t *d) {
    if (!idx) return PG_ERR_INVALID_ARG;
    if (params) *params = idx->params;
    if (d) *d = idx->d;
    return PG_OK;
}

extern "C" pg_status pg_index_save(pg_ctx *ctx, const pg_index *idx, const char *path) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!idx || !path) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    if ((int)idx->layers.size() > kMaxLayers)
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "index has more than %d layers", kMaxLayers);
    FileHeader h;
    h.n = idx->n;
    h.d = idx->d;
    h.metric = (int32_t)idx->metric;
    h.ep_top = idx->ep_top;
    h.ep_base = idx->ep_base;
    h.p = idx->params;
    h.layers = (int32_t)idx->layers.size();
    for (int i = 0; i < h.layers; ++i) {
        h.count[i] = idx->layers[(size_t)i].count;
        h.R[i] = idx->layers[(size_t)i].R;
        h.has_gid[i] = idx->layers[(size_t)i].gid ? 1 : 0;
    }
    PG_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const std::string tmp = std::string(path) + ".partial";
    Writer w;
    w.f = fopen(tmp.c_str(), "wb");
    if (!w.f) return pg_fail(ctx, PG_ERR_IO, "pg_index_save: cannot create %s: %s", tmp.c_str(),
                             strerror(errno));
    auto abandon = [&](pg_status st, const char *what) {
        fclose(w.f);
        remove(tmp.c_str());
        return st == PG_ERR_IO ? pg_fail(ctx, st, "pg_index_save: %s", what) : st;
    };
    write_header(w, h);
    std::vector<int32_t> buf;
    for (int i = 0; w.ok && i < h.layers; ++i) {
        const pg_layer &l = idx->layers[(size_t)i];
        const int32_t *parts[3] = {l.gid, l.deg, l.nbr};
        const int64_t sizes[3] = {l.gid ? l.count : 0, l.count, l.count * l.R};
        for (int k = 0; k < 3 && w.ok; ++k) {
            if (!sizes[k]) continue;
            buf.resize((size_t)sizes[k]);
            cudaError_t e = cudaMemcpy(buf.data(), parts[k], (size_t)sizes[k] * 4,
                                       cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return abandon(pg_cuda_fail(ctx, e, "pg_index_save copy"), "");
            w.put(buf.data(), (size_t)sizes[k] * 4);
        }
    }
    const int64_t per = std::max<int64_t>(1, (int64_t)(kChunk / ((size_t)h.d * 4)));
    std::vector<float> pts((size_t)(std::min(per, h.n) * h.d));
    for (int64_t r0 = 0; w.ok && r0 < h.n; r0 += per) {
        const int64_t rows = std::min(per, h.n - r0);
        cudaError_t e = cudaMemcpy(pts.data(), idx->D + r0 * h.d, (size_t)(rows * h.d) * 4,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return abandon(pg_cuda_fail(ctx, e, "pg_index_save copy"), "");
        w.put(pts.data(), (size_t)(rows * h.d) * 4);
    }
    if (!w.ok) return abandon(PG_ERR_IO, "write failed");
    const uint64_t sum = w.hash.finish();
    if (fwrite(&sum, 1, 8, w.f) != 8) return abandon(PG_ERR_IO, "write failed");
    if (fclose(w.f) != 0) {
        remove(tmp.c_str());
        return pg_fail(ctx, PG_ERR_IO, "pg_index_save: close failed");
    }
    if (rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return pg_fail(ctx, PG_ERR_IO, "pg_index_save: cannot rename to %s: %s", path,
                       strerror(errno));
    }
    return PG_OK;
}

extern "C" pg_status pg_index_load(pg_ctx *ctx, const char *path, pg_index **out) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!path || !out) return pg_fail(ctx, PG_ERR_INVALID_ARG, "null pointer");
    *out = nullptr;
    pg_index *idx = new (std::nothrow) pg_index();
    if (!idx) return pg_fail(ctx, PG_ERR_OOM, "host allocation");
    FileHeader h;
    std::string msg;
    pg_status cuda_st = PG_OK;
    auto on_layer = [&](int i, LayerHost &L) {
        if (i == 0) {
            idx->n = h.n;
            idx->d = h.d;
            idx->metric = (pg_metric)h.metric;
            idx->ep_top = h.ep_top;
            idx->ep_base = h.ep_base;
            idx->params = h.p;
            idx->layers.resize((size_t)h.layers);
            if (cudaMalloc(&idx->owned, (size_t)(h.n * h.d) * 4) != cudaSuccess) {
                idx->owned = nullptr;
                cuda_st = pg_fail(ctx, PG_ERR_CUDA, "pg_index_load: allocation of the points");
                return false;
            }
            idx->D = idx->owned;
            idx->capacity = h.n;
        }
        pg_layer &l = idx->layers[(size_t)i];
        l.count = l.cap = h.count[i];
        l.R = h.R[i];
        pg_status st = upload(ctx, l.deg, L.deg);
        if (st == PG_OK) st = upload(ctx, l.nbr, L.nbr);
        if (st == PG_OK && h.has_gid[i]) {
            std::vector<int32_t> rows((size_t)h.n, -1);
            for (size_t t = 0; t < L.gid.size(); ++t) rows[(size_t)L.gid[t]] = (int32_t)t;
            st = upload(ctx, l.gid, L.gid);
            if (st == PG_OK) st = upload(ctx, l.rows, rows);
            if (st == PG_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
                st = pg_fail(ctx, PG_ERR_CUDA, "pg_index_load: copy");
        } else if (st == PG_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            st = pg_fail(ctx, PG_ERR_CUDA, "pg_index_load: copy");
        }
        cuda_st = st;
        return st == PG_OK;
    };
    auto on_points = [&](const float *p, int64_t r0, int64_t rows) {
        if (cudaMemcpy(idx->owned + r0 * h.d, p, (size_t)(rows * h.d) * 4,
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            cuda_st = pg_fail(ctx, PG_ERR_CUDA, "pg_index_load: copy of the points");
            return false;
        }
        return true;
    };
    const pg_status st = parse_file(path, h, msg, on_layer, on_points);
    if (st != PG_OK) {
        delete idx;
        if (cuda_st != PG_OK) return cuda_st;
        return pg_fail(ctx, st, "%s", msg.c_str());
    }
    *out = idx;
    return PG_OK;
}

extern "C" pg_status pg_index_file_check(const char *path, int64_t *n, int32_t *d,
                                         int32_t *n_layers, char *msg, size_t msg_len) {
    if (msg && msg_len) msg[0] = '\0';
    if (!path) return PG_ERR_INVALID_ARG;
    FileHeader h;
    std::string why;
    const pg_status st = parse_file(path, h, why, nullptr, nullptr);
    if (st != PG_OK) {
        if (msg && msg_len) snprintf(msg, msg_len, "%s", why.c_str());
        return st;
    }
    if (n) *n = h.n;
    if (d) *d = h.d;
    if (n_layers) *n_layers = h.layers;
    return PG_OK;
}
