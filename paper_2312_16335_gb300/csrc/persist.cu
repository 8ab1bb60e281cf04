// Index files: leanvec_index_save / leanvec_index_load / leanvec_index_file_check.
//
// One file holds what a search needs: the metric, the sizes, the primary store (LVQ-4 / LVQ-8
// records and their mean, or float32 records), the secondary store (LVQ-8 records and their mean,
// or FP16 records), the graph and its entry point.  Layout (little-endian, fixed 96-byte header):
//   0  char[8] "LEANVEC"    8  u32 version = 1     12 u32 header bytes = 96
//   16 i32 metric   20 i32 D   24 i32 d   28 i32 primary bits   32 i32 secondary bits
//   36 i32 R        40 i32 entry            44 f32 mu2
//   48 i64 n        56 i64 primary stride   64 i64 secondary stride   72 three zero i64
//   96 primary records (n x primary stride bytes); primary mean (d float32, LVQ primaries only);
//      secondary records (n x secondary stride bytes, when there is a secondary store);
//      secondary mean (D float32, LVQ-8 secondaries only); graph (n x R int32, when R > 0)
//   end: u64 checksum of every preceding byte: 64-bit FNV-1a over the little-endian 64-bit
//        words of that byte stream, zero-padded to a multiple of 8 bytes.
// A file is validated completely (sizes, strides against the record geometry, checksum, graph ids)
// before anything is written to the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "index.cuh"

namespace lv {

int launch_graph_sanitize(int32_t *graph, int64_t n, int R, int *status, cudaStream_t st);

constexpr char FILE_MAGIC[8] = {'L', 'E', 'A', 'N', 'V', 'E', 'C', 0};
constexpr uint32_t FILE_VERSION = 1, HEADER_BYTES = 96;

struct FileHeader {
    int32_t metric = 0, D = 0, d = 0, pbits = 0, sbits = 0, R = 0, entry = -1;
    float mu2 = 0.f;
    int64_t n = 0, pstride = 0, sstride = 0;
};

// 64-bit FNV-1a over 64-bit little-endian words, fed in arbitrary pieces
struct WordFnv {
    uint64_t h = 0xcbf29ce484222325ull;
    uint8_t part[8] = {};
    int np = 0;
    void word(uint64_t w) { h = (h ^ w) * 0x100000001b3ull; }
    void update(const void *p, size_t len) {
        const uint8_t *b = static_cast<const uint8_t *>(p);
        while (len && np) {
            part[np++] = *b++;
            --len;
            if (np == 8) {
                uint64_t w;
                std::memcpy(&w, part, 8);
                word(w);
                np = 0;
            }
        }
        for (; len >= 8; len -= 8, b += 8) {
            uint64_t w;
            std::memcpy(&w, b, 8);
            word(w);
        }
        if (len) {  // fewer than 8 bytes left, and no partial word pending
            std::memcpy(part, b, len);
            np = (int)len;
        }
    }
    uint64_t final() {
        if (np) {
            std::memset(part + np, 0, 8 - np);
            uint64_t w;
            std::memcpy(&w, part, 8);
            word(w);
            np = 0;
        }
        return h;
    }
};

static void put32(uint8_t *b, int off, uint32_t v) { std::memcpy(b + off, &v, 4); }
static void put64(uint8_t *b, int off, uint64_t v) { std::memcpy(b + off, &v, 8); }
static uint32_t get32(const uint8_t *b, int off) {
    uint32_t v;
    std::memcpy(&v, b + off, 4);
    return v;
}
static uint64_t get64(const uint8_t *b, int off) {
    uint64_t v;
    std::memcpy(&v, b + off, 8);
    return v;
}

static void encode_header(const FileHeader &h, uint8_t *b) {
    std::memset(b, 0, HEADER_BYTES);
    std::memcpy(b, FILE_MAGIC, 8);
    put32(b, 8, FILE_VERSION);
    put32(b, 12, HEADER_BYTES);
    put32(b, 16, (uint32_t)h.metric);
    put32(b, 20, (uint32_t)h.D);
    put32(b, 24, (uint32_t)h.d);
    put32(b, 28, (uint32_t)h.pbits);
    put32(b, 32, (uint32_t)h.sbits);
    put32(b, 36, (uint32_t)h.R);
    put32(b, 40, (uint32_t)h.entry);
    uint32_t m;
    std::memcpy(&m, &h.mu2, 4);
    put32(b, 44, m);
    put64(b, 48, (uint64_t)h.n);
    put64(b, 56, (uint64_t)h.pstride);
    put64(b, 64, (uint64_t)h.sstride);
}

// section sizes in bytes, in file order
struct Sections {
    int64_t prim = 0, pmean = 0, sec = 0, smean = 0, graph = 0;
    int64_t total() const { return prim + pmean + sec + smean + graph; }
};

static Sections sections_of(const FileHeader &h) {
    Sections s;
    s.prim = h.n * h.pstride;
    s.pmean = h.pbits == 32 ? 0 : 4 * (int64_t)h.d;
    s.sec = h.sbits ? h.n * h.sstride : 0;
    s.smean = h.sbits == 8 ? 4 * (int64_t)h.D : 0;
    s.graph = 4 * h.n * (int64_t)h.R;
    return s;
}

// header fields against each other and the record geometry
static int check_header(const FileHeader &h) {
    auto bad = [](const char *what) { return fail(LV_ERR_CORRUPT, std::string("index file: ") + what); };
    if (h.metric != LV_METRIC_IP && h.metric != LV_METRIC_L2) return bad("unknown metric");
    if (h.n < 1 || h.n >= (int64_t)0x7fffffff) return bad("n out of range");
    if (h.D < 1 || h.D > (1 << 20) || h.d < 1 || h.d > h.D) return bad("dimensions out of range");
    if (h.pbits != 4 && h.pbits != 8 && h.pbits != 32) return bad("primary bits must be 4, 8 or 32");
    if (h.sbits != 0 && h.sbits != 8 && h.sbits != 16) return bad("secondary bits must be 0, 8 or 16");
    if (h.pbits == 32 && (h.d != h.D || h.sbits != 0)) return bad("a float32 store has d = D and no secondaries");
    if (h.R < 0 || h.R > RMAX) return bad("R out of range");
    if (h.R == 0 ? h.entry != -1 : (h.entry < 0 || h.entry >= h.n)) return bad("entry out of range");
    RecGeom pg, sg;
    rec_geom(h.d, h.pbits, pg, h.metric);
    if (pg.stride != h.pstride) return bad("primary stride does not match the record geometry");
    if (h.sbits) {
        rec_geom(h.D, h.sbits, sg, h.metric);
        if (sg.stride != h.sstride) return bad("secondary stride does not match the record geometry");
    } else if (h.sstride != 0) {
        return bad("secondary stride without a secondary store");
    }
    return LV_OK;
}

// the whole file, validated: header, sizes, checksum, graph ids
struct FileImage {
    FileHeader h;
    std::vector<uint8_t> body;  // the sections, in file order
};

static int read_index_file(const char *path, FileImage &img) {
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(LV_ERR_ARG, std::string("index file: cannot open ") + path);
    uint8_t hb[HEADER_BYTES];
    int rc = LV_OK;
    int64_t size = -1;
    if (std::fseek(f, 0, SEEK_END) == 0) size = (int64_t)std::ftell(f);
    if (size < (int64_t)HEADER_BYTES + 8 || std::fseek(f, 0, SEEK_SET) != 0 ||
        std::fread(hb, 1, HEADER_BYTES, f) != HEADER_BYTES) {
        std::fclose(f);
        return fail(LV_ERR_CORRUPT, "index file: shorter than a header");
    }
    if (std::memcmp(hb, FILE_MAGIC, 8) != 0 || get32(hb, 8) != FILE_VERSION || get32(hb, 12) != HEADER_BYTES) {
        std::fclose(f);
        return fail(LV_ERR_CORRUPT, "index file: not a version-1 leanvec index file");
    }
    FileHeader &h = img.h;
    h.metric = (int32_t)get32(hb, 16);
    h.D = (int32_t)get32(hb, 20);
    h.d = (int32_t)get32(hb, 24);
    h.pbits = (int32_t)get32(hb, 28);
    h.sbits = (int32_t)get32(hb, 32);
    h.R = (int32_t)get32(hb, 36);
    h.entry = (int32_t)get32(hb, 40);
    uint32_t m = get32(hb, 44);
    std::memcpy(&h.mu2, &m, 4);
    h.n = (int64_t)get64(hb, 48);
    h.pstride = (int64_t)get64(hb, 56);
    h.sstride = (int64_t)get64(hb, 64);
    rc = check_header(h);
    const Sections s = rc == LV_OK ? sections_of(h) : Sections();
    if (rc == LV_OK && size != (int64_t)HEADER_BYTES + s.total() + 8)
        rc = fail(LV_ERR_CORRUPT, "index file: size does not match its header");
    uint8_t cb[8];
    if (rc == LV_OK) {
        img.body.resize((size_t)s.total());
        if (std::fread(img.body.data(), 1, img.body.size(), f) != img.body.size() || std::fread(cb, 1, 8, f) != 8)
            rc = fail(LV_ERR_CORRUPT, "index file: read failed");
    }
    std::fclose(f);
    if (rc != LV_OK) return rc;
    WordFnv fnv;
    fnv.update(hb, HEADER_BYTES);
    fnv.update(img.body.data(), img.body.size());
    if (fnv.final() != get64(cb, 0)) return fail(LV_ERR_CORRUPT, "index file: checksum mismatch");
    const int32_t *g = reinterpret_cast<const int32_t *>(img.body.data() + (s.total() - s.graph));
    for (int64_t i = 0; i < h.n * h.R; ++i)
        if (g[i] < -1 || g[i] >= h.n) return fail(LV_ERR_CORRUPT, "index file: graph id out of range");
    return LV_OK;
}

static void info_of(const FileHeader &h, lv_index_info *out) {
    std::memset(out, 0, sizeof(*out));
    out->n = h.n;
    out->D = h.D;
    out->d = h.d;
    out->primary_bits = h.pbits;
    out->secondary_bits = h.sbits;
    out->primary_stride = h.pstride;
    out->secondary_stride = h.sstride;
    out->R = h.R;
    out->entry = h.entry;
    out->mu2 = h.mu2;
}

}  // namespace lv

using namespace lv;

extern "C" {

int leanvec_index_file_check(const char *path, lv_index_info *out) {
    if (!path) return fail(LV_ERR_ARG, "index_file_check: null path");
    FileImage img;
    int rc = read_index_file(path, img);
    if (rc == LV_OK && out) info_of(img.h, out);
    return rc;
}

int leanvec_index_save(const lv_index *idx, const char *path, lv_stream_t stream) {
    if (!idx || !path) return fail(LV_ERR_ARG, "index_save: null argument");
    if (idx->n == 0 || !idx->prim) return fail(LV_ERR_STATE, "index_save: the index has no store");
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "index_save: cannot select device");
    LV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    FileHeader h;
    h.metric = idx->metric;
    h.D = idx->D;
    h.d = idx->d;
    h.pbits = idx->pbits;
    h.sbits = idx->sec ? idx->sbits : 0;
    h.R = idx->graph ? idx->R : 0;
    h.entry = h.R ? idx->entry : -1;
    h.mu2 = idx->mu2;
    h.n = idx->n;
    h.pstride = idx->pg.stride;
    h.sstride = h.sbits ? idx->sg.stride : 0;
    const Sections s = sections_of(h);
    uint8_t hb[HEADER_BYTES];
    encode_header(h, hb);
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(LV_ERR_ARG, std::string("index_save: cannot create ") + path);
    WordFnv fnv;
    bool ok = std::fwrite(hb, 1, HEADER_BYTES, f) == HEADER_BYTES;
    fnv.update(hb, HEADER_BYTES);
    std::vector<uint8_t> buf;
    const int64_t CH = (int64_t)64 << 20;
    auto dump = [&](const void *dev, int64_t bytes) -> int {
        for (int64_t o = 0; ok && o < bytes; o += CH) {
            const int64_t len = std::min(CH, bytes - o);
            buf.resize((size_t)len);
            if (cudaMemcpy(buf.data(), static_cast<const uint8_t *>(dev) + o, (size_t)len, cudaMemcpyDeviceToHost) !=
                cudaSuccess)
                return fail(LV_ERR_CUDA, "index_save: device copy failed");
            fnv.update(buf.data(), (size_t)len);
            ok = std::fwrite(buf.data(), 1, (size_t)len, f) == (size_t)len;
        }
        return LV_OK;
    };
    int rc = dump(idx->prim, s.prim);
    if (rc == LV_OK && s.pmean) rc = dump(idx->pmean, s.pmean);
    if (rc == LV_OK && s.sec) rc = dump(idx->sec, s.sec);
    if (rc == LV_OK && s.smean) rc = dump(idx->smean, s.smean);
    if (rc == LV_OK && s.graph) rc = dump(idx->graph, s.graph);
    if (rc == LV_OK) {
        uint8_t cb[8];
        put64(cb, 0, fnv.final());
        ok = ok && std::fwrite(cb, 1, 8, f) == 8;
    }
    ok = (std::fclose(f) == 0) && ok;
    if (rc == LV_OK && !ok) rc = fail(LV_ERR_ARG, std::string("index_save: write failed for ") + path);
    return rc;
}

int leanvec_index_load(lv_index *idx, const char *path, lv_stream_t stream) {
    if (!idx || !path) return fail(LV_ERR_ARG, "index_load: null argument");
    FileImage img;
    int rc = read_index_file(path, img);
    if (rc != LV_OK) return rc;
    DeviceGuard g(idx->device);
    if (!g.ok) return fail(LV_ERR_CUDA, "index_load: cannot select device");
    cudaStream_t st = (cudaStream_t)stream;
    const FileHeader &h = img.h;
    const Sections s = sections_of(h);
    index_free_stores(idx);
    idx->metric = h.metric;
    const uint8_t *p = img.body.data();
    auto upload = [&](void **dev, int64_t bytes) -> int {
        if (!bytes) return LV_OK;
        if (cudaMalloc(dev, (size_t)bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(LV_ERR_OOM, "index_load: device allocation failed");
        }
        if (cudaMemcpy(*dev, p, (size_t)bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(LV_ERR_CUDA, "index_load: device copy failed");
        p += bytes;
        return LV_OK;
    };
    rc = upload((void **)&idx->prim, s.prim);
    if (rc == LV_OK) rc = upload((void **)&idx->pmean, s.pmean);
    if (rc == LV_OK) rc = upload((void **)&idx->sec, s.sec);
    if (rc == LV_OK) rc = upload((void **)&idx->smean, s.smean);
    if (rc == LV_OK) rc = upload((void **)&idx->graph, s.graph);
    if (rc == LV_OK && h.R) rc = launch_graph_sanitize(idx->graph, h.n, h.R, idx->status, st);
    if (rc == LV_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(LV_ERR_CUDA, "index_load: sync failed");
    if (rc != LV_OK) {
        index_free_stores(idx);
        return rc;
    }
    idx->n = h.n;
    idx->D = h.D;
    idx->d = h.d;
    idx->pbits = h.pbits;
    idx->sbits = h.sbits;
    rec_geom(h.d, h.pbits, idx->pg, h.metric);
    if (h.sbits) rec_geom(h.D, h.sbits, idx->sg, h.metric);
    idx->mu2 = h.mu2;
    idx->R = h.R;
    idx->entry = h.entry;
    return LV_OK;
}

}  // extern "C"
