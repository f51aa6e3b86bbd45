// Plan cache files: a built plan (host tables and every device array) written
// to disk and read back, so that a plan whose build takes a minute or more
// (Nside = 2048, L = 4096) loads in the time it takes to read it.  The paper
// keeps its precomputed data in files too and excludes their load time from
// its timings; so do we.
//
// Layout: a fixed header (magic, format version, the plan key including the
// spin, payload size, FNV-1a 64 checksum of the payload), then one payload per
// operator (two for a polarised plan, F+ then F-): the plan's scalars and
// host vectors, every device array in allocation order, and the device
// pointers of the plan as indices into that array list.  A load checks the
// magic, version, key, sizes and checksum before the plan is used; any
// mismatch is SHTB_ECORRUPT, an unreadable file SHTB_EIO.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "shtb_butterfly.h"
#include "shtb_internal.h"

namespace {

constexpr char kMagic[8] = {'S', 'H', 'T', 'B', 'P', 'L', 'A', 'N'};
constexpr uint32_t kVersion = 4;

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int32_t nside, lmax, leaf_cols, max_depth;
    int32_t spin, reserved;          // 0 scalar, 2 polarised (two plan payloads: F+ then F-)
    double eps, rho;
    uint64_t payload_bytes;
    uint64_t checksum;
};

struct Fnv {
    uint64_t h = 1469598103934665603ULL;
    void add(const void *p, size_t n)
    {
        const unsigned char *c = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ULL;
        }
    }
};

struct Writer {
    FILE *f;
    Fnv sum;
    uint64_t bytes = 0;
    bool ok = true;
    void raw(const void *p, size_t n)
    {
        if (!ok || n == 0) return;
        ok = fwrite(p, 1, n, f) == n;
        sum.add(p, n);
        bytes += n;
    }
    template <class T> void val(const T &v) { raw(&v, sizeof(T)); }
    template <class T> void vec(const std::vector<T> &v)
    {
        const uint64_t n = v.size();
        val(n);
        raw(v.data(), sizeof(T) * v.size());
    }
};

struct Reader {
    FILE *f;
    Fnv sum;
    uint64_t bytes = 0, limit = 0;
    bool ok = true;
    void raw(void *p, size_t n)
    {
        if (!ok || n == 0) return;
        if (bytes + n > limit) { ok = false; return; }
        ok = fread(p, 1, n, f) == n;
        if (ok) sum.add(p, n);
        bytes += n;
    }
    template <class T> void val(T &v) { raw(&v, sizeof(T)); }
    template <class T> void vec(std::vector<T> &v, uint64_t max_n)
    {
        uint64_t n = 0;
        val(n);
        if (!ok || n > max_n) { ok = false; return; }
        v.resize(n);
        raw(v.data(), sizeof(T) * n);
    }
};

// the device pointers of a plan, as pointers to the fields that hold them
std::vector<const void **> pointer_fields(shtb_plan_s *p)
{
    PlanView &v = p->view;
    std::vector<const void **> f = {
        (const void **)&v.coef, (const void **)&v.xarg, (const void **)&v.xform, (const void **)&v.jstart,
        (const void **)&v.vstart, (const void **)&v.ring_J, (const void **)&v.ring_s,
        (const void **)&v.ring_start, (const void **)&v.ring_tw, (const void **)&v.tw,
        (const void **)&v.ring_rad, (const void **)&v.rad, (const void **)&v.ring_mx,
        (const void **)&v.ring_mfb, (const void **)&v.mfb, (const void **)&v.ring_mtw, (const void **)&v.mtw,
        (const void **)&v.ring_ab, (const void **)&v.ab, (const void **)&v.ring_rdr, (const void **)&v.rdr,
        (const void **)&v.rdr_int, (const void **)&v.rdr_dbl,
        (const void **)&p->d_direct_rings, (const void **)&p->d_blue_rings, (const void **)&p->d_big_rings,
        (const void **)&p->d_chunk_list};
    if (p->bf) {
        BfPlanDev &bf = *p->bf;
        for (const void **q : {(const void **)&bf.ritems, (const void **)&bf.rgroups, (const void **)&bf.ints,
                               (const void **)&bf.dbl, (const void **)&bf.depth_parity})
            f.push_back(q);
        for (auto &li : bf.level_items) f.push_back((const void **)&li);
    }
    return f;
}

bool key_matches(const Header &h, const shtb_plan_s *p)
{
    return h.nside == p->nside && h.lmax == p->lmax && h.eps == p->eps && h.leaf_cols == p->opts.leaf_cols &&
           h.max_depth == p->opts.max_depth && h.rho == p->opts.rho && h.spin == p->opts.spin;
}

// one plan's payload: scalars, host vectors, device arrays, pointer indices
bool write_payload(Writer &w, shtb_plan_s *p)
{
    w.val(p->nrings); w.val(p->nhalf); w.val(p->npix); w.val(p->nalm); w.val(p->kind);
    w.val(p->max_K_direct); w.val(p->max_M_mx); w.val(p->max_K_big);
    w.val(p->blue_split); w.val(p->max_M_small);
    w.val(p->chunk_kind); w.val(p->chunk_pix); w.val(p->stats);
    w.vec(p->ring_J); w.vec(p->ring_s); w.vec(p->ring_start);
    w.vec(p->direct_rings); w.vec(p->blue_rings); w.vec(p->big_rings);
    w.val(p->view);                                      // scalars; pointers are remapped below
    const int compressed = p->bf ? 1 : 0;
    w.val(compressed);
    if (p->bf) {
        const BfPlanDev &bf = *p->bf;
        w.val(bf.depth_max); w.val(bf.n_ritems); w.val(bf.n_rgroups);
        w.vec(bf.level_counts); w.vec(bf.level_maxnc);
        w.val(bf.u_entries); w.val(bf.qt_entries); w.val(bf.n_dense); w.val(bf.n_r); w.val(bf.n_ident);
    }
    // device arrays, in allocation order, staged through a host buffer
    const uint64_t na = p->allocations.size();
    w.val(na);
    std::vector<char> buf;
    for (size_t i = 0; i < p->allocations.size() && w.ok; ++i) {
        const uint64_t n = p->alloc_bytes[i];
        w.val(n);
        buf.resize(n);
        if (cudaMemcpy(buf.data(), p->allocations[i], n, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
        w.raw(buf.data(), n);
    }
    // the plan's device pointers as allocation indices (0 = null)
    for (const void **fp : pointer_fields(p)) {
        uint64_t idx = 0;
        for (size_t i = 0; i < p->allocations.size(); ++i)
            if (p->allocations[i] == *fp) idx = i + 1;
        w.val(idx);
    }
    return true;
}

// Fills p (device, opts and key already set) from one payload; returns
// SHTB_OK with r.ok telling whether the bytes were well formed, or an
// allocation error.
int read_payload(Reader &r, shtb_plan_s *p)
{
    const uint64_t big = 1ULL << 40;
    int kind = -1;
    r.val(p->nrings); r.val(p->nhalf); r.val(p->npix); r.val(p->nalm); r.val(kind);
    if (r.ok && kind != p->kind) r.ok = false;
    r.val(p->max_K_direct); r.val(p->max_M_mx); r.val(p->max_K_big);
    r.val(p->blue_split); r.val(p->max_M_small);
    r.val(p->chunk_kind); r.val(p->chunk_pix);
    shtb_plan_stats_t st{};          // set once the uploads (which count their bytes) are done
    r.val(st);
    r.vec(p->ring_J, big); r.vec(p->ring_s, big); r.vec(p->ring_start, big);
    r.vec(p->direct_rings, big); r.vec(p->blue_rings, big); r.vec(p->big_rings, big);
    if (r.ok && (p->blue_split < 0 || p->blue_split > (int)p->blue_rings.size())) r.ok = false;
    for (const auto &row : p->chunk_kind)
        for (const auto &ck : row)
            if (ck.n < 0 || ck.off < 0 || ck.split < 0 || ck.split > ck.n) r.ok = false;
    r.val(p->view);
    int compressed = 0;
    r.val(compressed);
    if (r.ok && compressed) {
        p->bf = new BfPlanDev();
        BfPlanDev &bf = *p->bf;
        r.val(bf.depth_max); r.val(bf.n_ritems); r.val(bf.n_rgroups);
        r.vec(bf.level_counts, 64); r.vec(bf.level_maxnc, 64);
        r.val(bf.u_entries); r.val(bf.qt_entries); r.val(bf.n_dense); r.val(bf.n_r); r.val(bf.n_ident);
        if (r.ok && (bf.depth_max < 0 || bf.depth_max > 64 || (int)bf.level_counts.size() != bf.depth_max))
            r.ok = false;
        if (r.ok) bf.level_items.assign(bf.depth_max, nullptr);
    }
    uint64_t na = 0;
    r.val(na);
    if (na > 4096) r.ok = false;
    std::vector<char> buf;
    for (uint64_t i = 0; i < na && r.ok; ++i) {
        uint64_t n = 0;
        r.val(n);
        if (!r.ok || n > r.limit - r.bytes) { r.ok = false; break; }
        buf.resize(n);
        r.raw(buf.data(), n);
        if (!r.ok) break;
        void *d = nullptr;
        const int rc = plan_alloc_upload(p, &d, buf.data(), n);
        if (rc) return rc;
    }
    for (const void **fp : pointer_fields(p)) {
        uint64_t idx = 0;
        r.val(idx);
        if (!r.ok || idx > p->allocations.size()) { r.ok = false; break; }
        *fp = idx ? p->allocations[idx - 1] : nullptr;
    }
    p->stats = st;
    return SHTB_OK;
}

}  // namespace

int plan_save(shtb_plan_s *p, const char *path)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return shtb_fail(SHTB_EIO, std::string("cannot create plan file ") + tmp);
    Header h{};
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = sizeof(Header);
    h.nside = p->nside;
    h.lmax = p->lmax;
    h.leaf_cols = p->opts.leaf_cols;
    h.max_depth = p->opts.max_depth;
    h.spin = p->opts.spin;
    h.eps = p->eps;
    h.rho = p->opts.rho;
    bool ok = fwrite(&h, sizeof h, 1, f) == 1;          // rewritten with the sizes at the end
    Writer w{f};
    bool dev_ok = write_payload(w, p);
    if (dev_ok && p->partner) dev_ok = write_payload(w, p->partner);
    if (!dev_ok) {
        fclose(f);
        remove(tmp.c_str());
        return shtb_fail(SHTB_ECUDA, "plan save: device copy failed");
    }
    h.payload_bytes = w.bytes;
    h.checksum = w.sum.h;
    ok = ok && w.ok && fseek(f, 0, SEEK_SET) == 0 && fwrite(&h, sizeof h, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return shtb_fail(SHTB_EIO, std::string("cannot write plan file ") + path);
    }
    return SHTB_OK;
}

// Fills a fresh plan (device, opts and key already set; for a polarised key,
// kind 1 with a fresh kind-2 partner) from a file.
int plan_load(shtb_plan_s *p, const char *path)
{
    FILE *f = fopen(path, "rb");
    if (!f) return shtb_fail(SHTB_EIO, std::string("cannot open plan file ") + path);
    Header h{};
    if (fread(&h, sizeof h, 1, f) != 1) {
        fclose(f);
        return shtb_fail(SHTB_ECORRUPT, std::string("plan file too short: ") + path);
    }
    if (memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion || h.header_bytes != sizeof(Header)) {
        fclose(f);
        return shtb_fail(SHTB_ECORRUPT, std::string("not a plan file of this version: ") + path);
    }
    if (!key_matches(h, p) || (h.spin == 2) != (p->partner != nullptr)) {
        fclose(f);
        return shtb_fail(SHTB_ECORRUPT, std::string("plan file is for another (nside, lmax, eps, options): ") + path);
    }
    Reader r{f};
    r.limit = h.payload_bytes;
    int rc = read_payload(r, p);
    if (!rc && r.ok && p->partner) rc = read_payload(r, p->partner);
    if (rc) {
        fclose(f);
        return rc;
    }
    const bool complete = r.ok && r.bytes == h.payload_bytes && fgetc(f) == EOF;
    fclose(f);
    if (!complete || r.sum.h != h.checksum)
        return shtb_fail(SHTB_ECORRUPT, std::string("plan file failed its size or checksum check: ") + path);
    return SHTB_OK;
}

std::string plan_cache_path(const shtb_plan_s *p, const char *dir)
{
    char name[256];
    snprintf(name, sizeof name, "shtb_plan_v%u_n%d_l%d_e%a_lc%d_md%d_r%a_s%d.bin", kVersion, p->nside, p->lmax,
             p->eps, p->opts.leaf_cols, p->opts.max_depth, p->opts.rho, p->opts.spin);
    std::string s(dir);
    if (!s.empty() && s.back() != '/') s += '/';
    return s + name;
}

int plan_read_key(const char *path, int *nside, int *lmax, double *eps, shtb_plan_opts *opts)
{
    FILE *f = fopen(path, "rb");
    if (!f) return shtb_fail(SHTB_EIO, std::string("cannot open plan file ") + path);
    Header h{};
    const bool got = fread(&h, sizeof h, 1, f) == 1;
    fclose(f);
    if (!got || memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion || h.header_bytes != sizeof(Header))
        return shtb_fail(SHTB_ECORRUPT, std::string("not a plan file of this version: ") + path);
    *nside = h.nside;
    *lmax = h.lmax;
    *eps = h.eps;
    opts->leaf_cols = h.leaf_cols;
    opts->max_depth = h.max_depth;
    opts->rho = h.rho;
    opts->spin = h.spin;
    return SHTB_OK;
}
