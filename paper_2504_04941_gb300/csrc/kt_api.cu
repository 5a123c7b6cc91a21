// kt_api.cu -- host side of libkt: network parsing, device tables, state buffers and
// the C entry points declared in include/kt.h.
#include <cuda_runtime.h>

#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "kt_internal.h"

using kt::NetView;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(KT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int align16(int x) { return (x + 15) & ~15; }

}  // namespace

void kt::set_error(const char *msg) { g_err = msg; }

// 2^(j/32) evaluated in long double and rounded once to double.
double kt::exp2_table(int j)
{
    return static_cast<double>(std::exp2(static_cast<long double>(j) / static_cast<long double>(kt::kExpTable)));
}

struct kt_network {
    std::string name;
    int ns = 0, ne = 0, nr = 0, energy = 0;
    double t_ref = 1.0, t_min = 1.0, t_max = 1e5;
    std::vector<double> mass, h, cv;
    std::vector<int> counts;                      // [ns*ne]
    std::vector<int> nin, nout;                   // [nr]
    std::vector<std::array<int, kt::kMaxSide>> in, out;
    std::vector<double> A, b, th;
    int cvpoly = 0;                               // heat capacities polynomial in T
    double t_mid = 0.0;
    std::vector<double> cvp;                      // [ns*10]: low-range then high-range coefficients
    std::vector<int> rtype;                       // [nr]: 0 Arrhenius, 1 tabulated, 2 photo
    std::vector<double> sig_r, sig_s;             // photo cross-sections per reaction / species
    int ntab = 0, tab_nT = 0, tab_nR = 0;
    double tab_T0 = 0, tab_T1 = 0, tab_R0 = 0, tab_R1 = 0;
    std::vector<int> tab_of;                      // [nr]: table row, -1 if none
    std::vector<double> tab;                      // [ntab][nR][nT] ln k
    std::vector<unsigned char> blob;
    NetView view{};
    const kt_mlp *mlp = nullptr;                  // attached learned-guess MLP (not owned)
    std::mutex mu;
    std::map<int, unsigned char *> dev_blob;      // device ordinal -> device copy

    ~kt_network()
    {
        int cur = 0;
        cudaGetDevice(&cur);
        for (auto &kv : dev_blob) {
            cudaSetDevice(kv.first);
            cudaFree(kv.second);
        }
        cudaSetDevice(cur);
    }

    // Device copy of the blob on the current device (uploaded once per device).
    int device_blob(const unsigned char **out)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        std::lock_guard<std::mutex> lk(mu);
        auto it = dev_blob.find(dev);
        if (it != dev_blob.end()) {
            *out = it->second;
            return KT_OK;
        }
        unsigned char *p = nullptr;
        e = cudaMalloc(&p, blob.size());
        if (e != cudaSuccess) return fail(KT_ENOMEM, "cudaMalloc(network tables): %s", cudaGetErrorString(e));
        e = cudaMemcpy(p, blob.data(), blob.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(p);
            return cuda_fail(e, "cudaMemcpy(network tables)");
        }
        dev_blob[dev] = p;
        *out = p;
        return KT_OK;
    }
};

struct kt_state {
    const kt_network *net = nullptr;
    long long ncells = 0;
    int device = 0;
    double *y = nullptr, *T = nullptr, *rho = nullptr;
    int *status = nullptr, *nsub = nullptr, *nnew = nullptr;
    kt::Scratch *scratch = nullptr;
    // captured integrate call (memset of the scratch + kernel), replayed while dt and
    // the options are unchanged
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;
    double g_dt = 0.0;
    kt_options g_opts{};
    kt_mlp *mlp = nullptr;                        // learned-guess MLP loaded for this state (owned)
    int *order = nullptr;                         // longest-first queue order (opts.schedule)
    unsigned *sched_work = nullptr;               // its histogram and cursors
};

namespace {

// ---------------------------------------------------------------- network file parser

struct Tok {
    std::istringstream in;
    explicit Tok(const std::string &s) : in(s) {}
    bool next(std::string &w) { return static_cast<bool>(in >> w); }
    bool word(const char *expect)
    {
        std::string w;
        return next(w) && w == expect;
    }
    bool integer(int &v)
    {
        std::string w;
        if (!next(w)) return false;
        char *end = nullptr;
        long x = std::strtol(w.c_str(), &end, 10);
        if (*end) return false;
        v = static_cast<int>(x);
        return true;
    }
    bool real(double &v)
    {
        std::string w;
        if (!next(w)) return false;
        char *end = nullptr;
        v = std::strtod(w.c_str(), &end);
        return *end == 0;
    }
};

std::string strip_comments(std::istream &f)
{
    std::string out, line;
    while (std::getline(f, line)) {
        auto p = line.find('#');
        if (p != std::string::npos) line.resize(p);
        out += line;
        out += '\n';
    }
    return out;
}

int parse_network(const std::string &text, kt_network *n)
{
    Tok t(text);
    int version = 0;
    std::string w;
    if (!(t.word("kratos_network") && t.integer(version) && version == 1))
        return fail(KT_EPARSE, "network: missing 'kratos_network 1' header");
    if (!(t.word("name") && t.next(n->name) && t.word("n_species") && t.integer(n->ns) &&
          t.word("n_elements") && t.integer(n->ne) && t.word("n_reactions") && t.integer(n->nr) &&
          t.word("energy") && t.integer(n->energy) && t.word("t_ref") && t.real(n->t_ref) &&
          t.word("t_min") && t.real(n->t_min) && t.word("t_max") && t.real(n->t_max) &&
          t.word("elements")))
        return fail(KT_EPARSE, "network: malformed header");
    if (n->ns < 1 || n->ns > 250 || n->ne < 1 || n->ne > kt::kMaxElements || n->nr < 0 ||
        (n->energy != 0 && n->energy != 1) || !(n->t_ref > 0) || !(n->t_min > 0) || !(n->t_max >= n->t_min))
        return fail(KT_EPARSE, "network: sizes or limits out of range");
    for (int e = 0; e < n->ne; ++e)
        if (!t.next(w)) return fail(KT_EPARSE, "network: element names");
    n->mass.resize(n->ns);
    n->h.resize(n->ns);
    n->cv.resize(n->ns);
    n->counts.resize(static_cast<size_t>(n->ns) * n->ne);
    for (int s = 0; s < n->ns; ++s) {
        if (!(t.word("species") && t.next(w) && t.real(n->mass[s]) && t.real(n->h[s]) && t.real(n->cv[s])))
            return fail(KT_EPARSE, "network: species line %d", s);
        for (int e = 0; e < n->ne; ++e)
            if (!t.integer(n->counts[s * n->ne + e])) return fail(KT_EPARSE, "network: species %d counts", s);
    }
    n->nin.resize(n->nr);
    n->nout.resize(n->nr);
    n->in.resize(n->nr);
    n->out.resize(n->nr);
    n->A.resize(n->nr);
    n->b.resize(n->nr);
    n->th.resize(n->nr);
    for (int r = 0; r < n->nr; ++r) {
        int pair = 0;
        n->in[r].fill(-1);
        n->out[r].fill(-1);
        if (!(t.word("reaction") && t.integer(n->nin[r]) && n->nin[r] >= 1 && n->nin[r] <= kt::kMaxSide))
            return fail(KT_EPARSE, "network: reaction %d reactants", r);
        for (int j = 0; j < n->nin[r]; ++j)
            if (!(t.integer(n->in[r][j]) && n->in[r][j] >= 0 && n->in[r][j] < n->ns))
                return fail(KT_EPARSE, "network: reaction %d reactant index", r);
        if (!(t.integer(n->nout[r]) && n->nout[r] >= 0 && n->nout[r] <= kt::kMaxSide))
            return fail(KT_EPARSE, "network: reaction %d products", r);
        for (int j = 0; j < n->nout[r]; ++j)
            if (!(t.integer(n->out[r][j]) && n->out[r][j] >= 0 && n->out[r][j] < n->ns))
                return fail(KT_EPARSE, "network: reaction %d product index", r);
        if (!(t.real(n->A[r]) && t.real(n->b[r]) && t.real(n->th[r]) && t.integer(pair)))
            return fail(KT_EPARSE, "network: reaction %d parameters", r);
    }
    // optional sections: heat capacities, photo-reactions, rate tables; then "end"
    n->rtype.assign(n->nr, 0);
    n->sig_r.assign(n->nr, 0.0);
    n->sig_s.assign(n->ns, 0.0);
    n->tab_of.assign(n->nr, -1);
    for (;;) {
        if (!t.next(w)) return fail(KT_EPARSE, "network: missing 'end'");
        if (w == "end") break;
        if (w == "cv_poly" && !n->cvpoly) {
            // cv_s(T) = sum_k a_k T^k below t_mid, sum_k b_k T^k from t_mid [J/(mol K)]
            if (!n->energy) return fail(KT_EPARSE, "network: cv_poly needs the temperature equation");
            if (!(t.real(n->t_mid) && n->t_mid > 0)) return fail(KT_EPARSE, "network: cv_poly t_mid");
            n->cvp.resize(static_cast<size_t>(n->ns) * 10);
            for (int s = 0; s < n->ns; ++s) {
                int sp = -1;
                if (!(t.word("cvp") && t.integer(sp) && sp == s)) return fail(KT_EPARSE, "network: cvp line %d", s);
                for (int k = 0; k < 10; ++k)
                    if (!t.real(n->cvp[s * 10 + k])) return fail(KT_EPARSE, "network: cvp %d coefficients", s);
            }
            n->cvpoly = 1;
        } else if (w == "photo") {
            // photo-reactions (Eq. photo-reaction-single): "ph <reaction> <sigma_r>", one reactant
            int np = -1;
            if (!(t.integer(np) && np >= 0 && np <= n->nr)) return fail(KT_EPARSE, "network: photo count");
            for (int i = 0; i < np; ++i) {
                int r = -1;
                double sg = -1.0;
                if (!(t.word("ph") && t.integer(r) && r >= 0 && r < n->nr && t.real(sg) && sg >= 0.0 &&
                      n->nin[r] == 1 && n->rtype[r] == 0))
                    return fail(KT_EPARSE, "network: photo-reaction line %d", i);
                n->rtype[r] = 2;
                n->sig_r[r] = sg;
                n->sig_s[n->in[r][0]] += sg;
            }
        } else if (w == "rate_table" && n->ntab == 0) {
            // ln k on log-spaced (T, rho) nodes per tabulated reaction (Sec. 2.2.1 item 3)
            if (!(t.integer(n->tab_nT) && t.real(n->tab_T0) && t.real(n->tab_T1) && t.integer(n->tab_nR) &&
                  t.real(n->tab_R0) && t.real(n->tab_R1) && t.integer(n->ntab)) ||
                n->tab_nT < 2 || n->tab_nT > 64 || n->tab_nR < 1 || n->tab_nR > 64 || n->ntab < 0 ||
                n->ntab > n->nr || !(n->tab_T0 > 0) || !(n->tab_T1 > n->tab_T0) || !(n->tab_R0 > 0) ||
                !(n->tab_nR == 1 || n->tab_R1 > n->tab_R0))
                return fail(KT_EPARSE, "network: rate_table grid");
            const int m = n->tab_nR * n->tab_nT;
            n->tab.assign(static_cast<size_t>(n->ntab) * m, 0.0);
            for (int i = 0; i < n->ntab; ++i) {
                int r = -1;
                if (!(t.word("tab") && t.integer(r) && r >= 0 && r < n->nr && n->rtype[r] == 0))
                    return fail(KT_EPARSE, "network: rate table %d", i);
                n->rtype[r] = 1;
                n->tab_of[r] = i;
                for (int q = 0; q < m; ++q)
                    if (!t.real(n->tab[static_cast<size_t>(i) * m + q]))
                        return fail(KT_EPARSE, "network: rate table %d values", i);
            }
        } else {
            return fail(KT_EPARSE, "network: unknown section '%s'", w.c_str());
        }
    }
    // element conservation of every reaction (Eq. method-const-elem)
    for (int r = 0; r < n->nr; ++r)
        for (int e = 0; e < n->ne; ++e) {
            int bal = 0;
            for (int j = 0; j < n->nin[r]; ++j) bal -= n->counts[n->in[r][j] * n->ne + e];
            for (int j = 0; j < n->nout[r]; ++j) bal += n->counts[n->out[r][j] * n->ne + e];
            if (bal != 0) return fail(KT_ENETWORK, "network: reaction %d does not conserve element %d", r, e);
        }
    return KT_OK;
}

// Pack the device tables (layout kt::NetView).
void build_blob(kt_network *n)
{
    NetView &v = n->view;
    v.ns = n->ns;
    v.ne = n->ne;
    v.nr = n->nr;
    v.energy = n->energy;
    v.N = n->ns + n->energy;
    v.t_ref = n->t_ref;
    v.t_min = n->t_min;
    v.t_max = n->t_max;
    int o = 0;
    v.off_A = o; o = align16(o + 8 * n->nr);
    v.off_b = o; o = align16(o + 8 * n->nr);
    v.off_th = o; o = align16(o + 8 * n->nr);
    v.off_h = o; o = align16(o + 8 * n->ns);
    v.off_cv = o; o = align16(o + 8 * n->ns);
    v.off_cnt = o; o = align16(o + 8 * n->ns * n->ne);
    v.off_idx = o; o = align16(o + 8 * n->nr);
    v.off_exp = o; o = align16(o + 8 * kt::kExpTable);
    // per-species lists of (reaction, +-1): a net coefficient nu appears as |nu| entries
    // of its sign, so every entry is one add (no per-lane branch on the coefficient)
    std::vector<int> rp(n->ns + 1, 0), re;
    for (int s = 0; s < n->ns; ++s) {
        rp[s] = static_cast<int>(re.size());
        for (int r = 0; r < n->nr; ++r) {
            int nu = 0;
            for (int j = 0; j < n->nout[r]; ++j) nu += n->out[r][j] == s;
            for (int j = 0; j < n->nin[r]; ++j) nu -= n->in[r][j] == s;
            for (int q = 0; q < (nu < 0 ? -nu : nu); ++q) re.push_back((r << 8) | ((nu < 0 ? -1 : 1) & 0xff));
        }
    }
    rp[n->ns] = static_cast<int>(re.size());
    v.nent = static_cast<int>(re.size());
    v.shape = n->nr > 0 ? 22 : 0;
    for (int r = 0; r < n->nr; ++r)
        if (n->nin[r] != 2 || n->nout[r] != 2) v.shape = 0;
    v.off_rp = o; o = align16(o + 4 * (n->ns + 1));
    v.off_re = o; o = align16(o + 4 * v.nent);
    v.cvpoly = n->cvpoly;
    v.t_mid = n->t_mid;
    v.off_cvp = o;
    if (n->cvpoly) o = align16(o + 8 * 10 * n->ns);
    // photo and table descriptors (staged with the rest); the tables themselves follow
    // the staged part and are read from global memory
    v.special = 0;
    v.nphoto = 0;
    for (int r = 0; r < n->nr; ++r) {
        if (n->rtype[r] != 0) v.special = 1;
        if (n->rtype[r] == 2) ++v.nphoto;
    }
    v.off_rtype = o; o = align16(o + 4 * n->nr);
    v.off_sigr = o; o = align16(o + 8 * n->nr);
    v.off_sigs = o; o = align16(o + 8 * n->ns);
    // the warp kernels stage the prefix up to here (the photo and table descriptors
    // only for networks that have such rates); the reaction heats serve the lane kernels
    v.bytes_warp = v.special ? o : v.off_rtype;
    v.off_dH = o; o = align16(o + 8 * n->nr);
    // FP32 copies of b, theta and the heats for the FP32 Jacobian of the lane kernels
    v.off_f32 = o; o = align16(o + 3 * 4 * n->nr);
    v.ntab = n->ntab;
    v.tab_nT = n->tab_nT;
    v.tab_nR = n->tab_nR;
    if (n->ntab) {
        v.tab_lt0 = std::log(n->tab_T0);
        v.tab_dlt = (std::log(n->tab_T1) - std::log(n->tab_T0)) / (n->tab_nT - 1);
        v.tab_lr0 = std::log(n->tab_R0);
        v.tab_dlr = n->tab_nR > 1 ? std::log(n->tab_R1) - std::log(n->tab_R0) : 1.0;
    }
    if (o < 16) o = 16;
    v.bytes = o;
    v.off_tab = o;
    o = align16(o + 8 * static_cast<int>(n->tab.size()));
    v.bytes_total = o;
    n->blob.assign(o, 0);
    auto put = [&](int off, int i, double x) { std::memcpy(n->blob.data() + off + 8 * i, &x, 8); };
    for (int r = 0; r < n->nr; ++r) {
        put(v.off_A, r, n->A[r]);
        put(v.off_b, r, n->b[r]);
        put(v.off_th, r, n->th[r]);
        double dH = 0.0;
        for (int j = 0; j < n->nout[r]; ++j) dH += n->h[n->out[r][j]];
        for (int j = 0; j < n->nin[r]; ++j) dH -= n->h[n->in[r][j]];
        put(v.off_dH, r, dH);
        const float f3[3] = {static_cast<float>(n->b[r]), static_cast<float>(n->th[r]), static_cast<float>(dH)};
        for (int q = 0; q < 3; ++q)
            std::memcpy(n->blob.data() + v.off_f32 + 4 * (q * n->nr + r), &f3[q], 4);
        unsigned char *ix = n->blob.data() + v.off_idx + 8 * r;
        bool distinct = true;   // no species twice among the reaction's reactants and products
        for (int a = 0; a < n->nin[r] + n->nout[r]; ++a)
            for (int b = a + 1; b < n->nin[r] + n->nout[r]; ++b) {
                const int sa = a < n->nin[r] ? n->in[r][a] : n->out[r][a - n->nin[r]];
                const int sb = b < n->nin[r] ? n->in[r][b] : n->out[r][b - n->nin[r]];
                if (sa == sb) distinct = false;
            }
        ix[0] = static_cast<unsigned char>(n->nin[r] | (distinct ? kt::kIdxDistinct : 0));
        ix[1] = static_cast<unsigned char>(n->nout[r]);
        for (int j = 0; j < kt::kMaxSide; ++j) {
            ix[2 + j] = static_cast<unsigned char>(j < n->nin[r] ? n->in[r][j] : kt::kIdxNone);
            ix[5 + j] = static_cast<unsigned char>(j < n->nout[r] ? n->out[r][j] : kt::kIdxNone);
        }
    }
    for (int j = 0; j < kt::kExpTable; ++j) put(v.off_exp, j, kt::exp2_table(j));
    std::memcpy(n->blob.data() + v.off_rp, rp.data(), 4 * rp.size());
    if (n->cvpoly) std::memcpy(n->blob.data() + v.off_cvp, n->cvp.data(), 8 * n->cvp.size());
    for (int r = 0; r < n->nr; ++r) {
        const int rt = n->rtype[r] == 1 ? (1 | (n->tab_of[r] << 8)) : n->rtype[r];
        std::memcpy(n->blob.data() + v.off_rtype + 4 * r, &rt, 4);
        put(v.off_sigr, r, n->sig_r[r]);
    }
    for (int s = 0; s < n->ns; ++s) put(v.off_sigs, s, n->sig_s[s]);
    if (!n->tab.empty()) std::memcpy(n->blob.data() + v.off_tab, n->tab.data(), 8 * n->tab.size());
    if (!re.empty()) std::memcpy(n->blob.data() + v.off_re, re.data(), 4 * re.size());
    for (int s = 0; s < n->ns; ++s) {
        put(v.off_h, s, n->h[s]);
        put(v.off_cv, s, n->cv[s]);
        for (int e = 0; e < n->ne; ++e) put(v.off_cnt, s * n->ne + e, static_cast<double>(n->counts[s * n->ne + e]));
    }
}

int check_opts(const kt_options *o)
{
    if (!o) return fail(KT_EINVAL, "options: NULL");
    if (!(o->rtol > 0) || !(o->atol > 0) || !(o->h_init > 0) || !(o->h_min >= 0) ||
        !(o->newton_rtol > 0) || !(o->newton_atol_frac > 0) || !(o->facmax >= 1) ||
        !(o->retry_h_factor > 0) || !(o->retry_facmax >= 1) || o->max_substeps < 1 ||
        o->max_newton < 1 || (o->form != KT_FORM_FP64 && o->form != KT_FORM_FP32LU) ||
        (o->guess != KT_GUESS_PREV && o->guess != KT_GUESS_MLP && o->guess != KT_GUESS_FULLSTEP) ||
        o->block_warps < 0 ||
        o->blocks_per_sm < 0 || (o->scheme != KT_SCHEME_BE && o->scheme != KT_SCHEME_TRBDF2) ||
        o->lane_variant < KT_LANE_AUTO || o->lane_variant > KT_LANE_LEAN)
        return fail(KT_EINVAL, "options: a field is out of range");
    if (o->scheme == KT_SCHEME_TRBDF2 && o->guess == KT_GUESS_MLP)
        return fail(KT_EINVAL, "options: the learned guess needs scheme KT_SCHEME_BE");
    return KT_OK;
}

kt::DevOpts dev_opts(const kt_options *o)
{
    kt::DevOpts d{};
    d.rtol = o->rtol;
    d.atol = o->atol;
    d.h_init = o->h_init;
    d.h_min = o->h_min;
    d.newton_rtol = o->newton_rtol;
    d.newton_atol_frac = o->newton_atol_frac;
    d.facmax = o->facmax;
    d.retry_h_factor = o->retry_h_factor;
    d.retry_facmax = o->retry_facmax;
    d.max_substeps = o->max_substeps;
    d.max_newton = o->max_newton;
    d.retry = o->retry;
    d.atol_mode = o->atol_mode;
    d.guess = o->guess;
    d.scheme = o->scheme;
    return d;
}

}  // namespace

extern "C" {

const char *kt_last_error(void) { return g_err.c_str(); }

int kt_options_default(kt_options *o)
{
    if (!o) return fail(KT_EINVAL, "kt_options_default: NULL");
    std::memset(o, 0, sizeof *o);
    o->rtol = 1e-6;
    o->atol = 1e-10;
    o->h_init = 1e-6;
    o->h_min = 1e-30;
    o->newton_rtol = 1e-12;
    o->newton_atol_frac = 1e-2;
    o->facmax = 4.0;
    o->retry_h_factor = 1e-3;
    o->retry_facmax = 2.0;
    o->max_substeps = 100000;
    o->max_newton = 8;
    o->form = KT_FORM_FP64;
    o->guess = KT_GUESS_PREV;
    o->persistent = 0;
    o->retry = 1;
    o->atol_mode = 0;
    return KT_OK;
}

int kt_network_load(const char *path, kt_network **out)
{
    if (!path || !out) return fail(KT_EINVAL, "kt_network_load: NULL argument");
    *out = nullptr;
    std::ifstream f(path);
    if (!f) return fail(KT_EPARSE, "kt_network_load: cannot open %s", path);
    kt_network *n = new (std::nothrow) kt_network();
    if (!n) return fail(KT_ENOMEM, "kt_network_load: out of memory");
    int rc = parse_network(strip_comments(f), n);
    if (rc != KT_OK) {
        delete n;
        return rc;
    }
    build_blob(n);
    *out = n;
    return KT_OK;
}

int kt_network_info(const kt_network *n, int *ns, int *ne, int *nr, int *energy)
{
    if (!n) return fail(KT_EINVAL, "kt_network_info: NULL network");
    if (ns) *ns = n->ns;
    if (ne) *ne = n->ne;
    if (nr) *nr = n->nr;
    if (energy) *energy = n->energy;
    return KT_OK;
}

void kt_network_free(kt_network *n) { delete n; }

size_t kt_scratch_bytes(void) { return sizeof(kt::Scratch); }

}  // extern "C"

namespace {

// Longest-first order of the state's cells from the Newton counts of the previous call
// (opts.schedule with a persistent launch); buffers are allocated on first use, outside
// any stream capture.  *order is null when the option is off.
int state_schedule(kt_state *st, const kt_options *opts, cudaStream_t s, bool launch, const int **order)
{
    *order = nullptr;
    if (!opts->schedule || !opts->persistent || st->ncells > 0x7fffffffLL) return KT_OK;
    if (!st->order || !st->sched_work) {
        cudaFree(st->order);
        cudaFree(st->sched_work);
        st->order = nullptr;
        st->sched_work = nullptr;
        cudaError_t e = cudaMalloc(&st->order, static_cast<size_t>(st->ncells) * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&st->sched_work, 2 * kt::kSchedBuckets * sizeof(unsigned));
        if (e != cudaSuccess) {
            cudaFree(st->order);
            cudaFree(st->sched_work);
            st->order = nullptr;
            st->sched_work = nullptr;
            return fail(KT_ENOMEM, "kt_integrate: schedule buffers: %s", cudaGetErrorString(e));
        }
    }
    if (launch) {
        const int ce = kt::launch_schedule(st->nnew, st->ncells, st->sched_work, st->order, s);
        if (ce != 0) return cuda_fail(static_cast<cudaError_t>(ce), "schedule kernels");
    }
    *order = st->order;
    return KT_OK;
}

int integrate_impl(const kt_network *net, int64_t ncells, const double *y_in, const double *T_in,
                   const double *rho, const double *dt_cell, double dt, const kt_options *opts, double *y_out,
                   double *T_out, int32_t *status, int32_t *n_substeps, int32_t *n_newton, void *scratch,
                   void *cuda_stream, const kt_mlp *mlp, const int *order = nullptr,
                   const double *flux = nullptr, const double *path = nullptr)
{
    if (!net) return fail(KT_EINVAL, "kt_integrate: NULL network");
    if (ncells < 0 || !(dt > 0) || !std::isfinite(dt)) return fail(KT_EINVAL, "kt_integrate: bad ncells or dt");
    int rc = check_opts(opts);
    if (rc) return rc;
    if (ncells == 0) return KT_OK;
    if (!y_in || !T_in || !y_out || !T_out || !scratch)
        return fail(KT_EINVAL, "kt_integrate_ptrs: NULL device buffer");
    if (reinterpret_cast<uintptr_t>(scratch) % 16) return fail(KT_EINVAL, "kt_integrate_ptrs: scratch not 16-B aligned");
    const int N = net->ns + net->energy;
    int cpw = opts->cells_per_warp;
    // tabulated and photo rates are evaluated by the warp-per-cell kernels
    if (cpw == 0) cpw = N <= kt::kLaneMaxN && !net->view.special ? 32 : 1;
    if ((cpw != 32 && cpw != 1) || (cpw == 32 && (N > kt::kLaneMaxN || net->view.special)))
        return fail(KT_EINVAL, "kt_integrate_ptrs: cells_per_warp %d not available for this network "
                               "(%d unknowns%s)", cpw, N, net->view.special ? ", tabulated or photo rates" : "");
    if (N > kt::kWarpMaxN)
        return fail(KT_EUNSUPPORTED, "kt_integrate_ptrs: %d unknowns per cell; this build handles up to %d", N,
                    kt::kWarpMaxN);
    kt_network *mn = const_cast<kt_network *>(net);
    const unsigned char *blob = nullptr;
    rc = mn->device_blob(&blob);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(kt::Scratch), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch)");
    kt::LaunchArgs a{};
    a.nv = net->view;
    a.blob = blob;
    a.o = dev_opts(opts);
    a.dt = dt;
    a.dt_cell = dt_cell;
    a.rho = rho;
    a.flux = flux;
    a.path = path;
    a.ncells = ncells;
    if (opts->guess == KT_GUESS_MLP) {
        const kt_mlp *m = mlp ? mlp : net->mlp;
        int dev = 0, cur = 0;
        a.mlp = kt::mlp_device_block(m, &a.mlp_nin, &a.mlp_nout, &dev);
        cudaGetDevice(&cur);
        if (!a.mlp) return fail(KT_EINVAL, "kt_integrate: learned guess requested but no MLP is loaded/attached");
        if (dev != cur) return fail(KT_EINVAL, "kt_integrate: the MLP lives on another device");
        if (a.mlp_nin != net->ns + 3 || a.mlp_nout != N)
            return fail(KT_EINVAL, "kt_integrate: MLP sizes (%d in, %d out) do not match the network (%d, %d)",
                        a.mlp_nin, a.mlp_nout, net->ns + 3, N);
        if (cpw != 32) return fail(KT_EUNSUPPORTED, "kt_integrate: the learned guess runs in the lane-per-cell kernels");
        if (!opts->persistent) return fail(KT_EUNSUPPORTED, "kt_integrate: the learned guess needs persistent=1");
    }
    a.y_in = y_in;
    a.T_in = T_in;
    a.y_out = y_out;
    a.T_out = T_out;
    a.status = status;
    a.nsub = n_substeps;
    a.nnew = n_newton;
    a.scratch = static_cast<kt::Scratch *>(scratch);
    a.order = opts->persistent ? order : nullptr;
    kt::LaunchCfg c{opts->form, opts->persistent, opts->block_warps, opts->blocks_per_sm, cpw, opts->lane_variant};
    int ce = cpw == 32 ? kt::launch_lane(a, c, cuda_stream) : kt::launch_warp(a, c, cuda_stream);
    if (ce != 0) return cuda_fail(static_cast<cudaError_t>(ce), "integrate kernel launch");
    return KT_OK;
}

}  // namespace

// Orthonormal basis of the row space of the element matrix N [n_elements][n_species]
// (modified Gram-Schmidt, two passes per vector; rows whose remainder falls below
// 1e-12 of their norm are dependent and dropped): Vr[s * rank + k].  P = I - Vr Vr^T is
// the projector onto the stoichiometric space null(N) (Sec. 2.1.3).
int kt::network_element_basis(const kt_network *net, double *Vr, int *ns_out, int *rank_out)
{
    if (!net) return fail(KT_EINVAL, "NULL network");
    const int ns = net->ns, ne = net->ne;
    if (ns > 256) return fail(KT_EUNSUPPORTED, "element basis: more than 256 species");
    std::vector<std::vector<double>> basis;
    for (int e = 0; e < ne; ++e) {
        std::vector<double> v(ns);
        double n0 = 0.0;
        for (int s = 0; s < ns; ++s) {
            v[s] = static_cast<double>(net->counts[s * ne + e]);
            n0 += v[s] * v[s];
        }
        n0 = std::sqrt(n0);
        if (!(n0 > 0.0)) continue;
        for (int pass = 0; pass < 2; ++pass)
            for (const auto &q : basis) {
                double d = 0.0;
                for (int s = 0; s < ns; ++s) d += q[s] * v[s];
                for (int s = 0; s < ns; ++s) v[s] -= d * q[s];
            }
        double nn = 0.0;
        for (int s = 0; s < ns; ++s) nn += v[s] * v[s];
        nn = std::sqrt(nn);
        if (!(nn > 1e-12 * n0)) continue;
        for (int s = 0; s < ns; ++s) v[s] /= nn;
        basis.push_back(v);
    }
    const int r = static_cast<int>(basis.size());
    for (int s = 0; s < ns; ++s)
        for (int k = 0; k < r; ++k) Vr[s * r + k] = basis[k][s];
    *ns_out = ns;
    *rank_out = r;
    return KT_OK;
}

int kt::prepare_launch(const kt_network *net, int64_t ncells, const double *y_in, const double *T_in,
                       const double *rho, double dt, const kt_options *opts, double *y_out, double *T_out,
                       int32_t *status, int32_t *n_substeps, int32_t *n_newton, kt::LaunchArgs *a,
                       kt::LaunchCfg *c, const unsigned char **host_blob)
{
    if (!net) return fail(KT_EINVAL, "NULL network");
    if (ncells < 0 || !(dt > 0) || !std::isfinite(dt)) return fail(KT_EINVAL, "bad ncells or dt");
    int rc = check_opts(opts);
    if (rc) return rc;
    if (opts->guess == KT_GUESS_MLP) return fail(KT_EUNSUPPORTED, "the learned guess is not available here");
    if (ncells > 0 && (!y_in || !T_in || !y_out || !T_out)) return fail(KT_EINVAL, "NULL device buffer");
    const int N = net->ns + net->energy;
    int cpw = opts->cells_per_warp;
    if (cpw == 0) cpw = N <= kt::kLaneMaxN && !net->view.special ? 32 : 1;
    if ((cpw != 32 && cpw != 1) || (cpw == 32 && (N > kt::kLaneMaxN || net->view.special)))
        return fail(KT_EINVAL, "cells_per_warp %d not available for this network (%d unknowns)", cpw, N);
    if (N > kt::kWarpMaxN) return fail(KT_EUNSUPPORTED, "%d unknowns per cell; this build handles up to %d", N, kt::kWarpMaxN);
    *a = kt::LaunchArgs{};
    a->nv = net->view;
    a->o = dev_opts(opts);
    a->dt = dt;
    a->rho = rho;
    a->ncells = ncells;
    a->y_in = y_in;
    a->T_in = T_in;
    a->y_out = y_out;
    a->T_out = T_out;
    a->status = status;
    a->nsub = n_substeps;
    a->nnew = n_newton;
    *c = kt::LaunchCfg{opts->form, opts->persistent, opts->block_warps, opts->blocks_per_sm, cpw, opts->lane_variant};
    *host_blob = net->blob.data();
    return KT_OK;
}

extern "C" {

int kt_integrate_ptrs(const kt_network *net, int64_t ncells, const double *y_in, const double *T_in,
                      const double *rho, double dt, const kt_options *opts, double *y_out,
                      double *T_out, int32_t *status, int32_t *n_substeps, int32_t *n_newton,
                      void *scratch, void *cuda_stream)
{
    return integrate_impl(net, ncells, y_in, T_in, rho, nullptr, dt, opts, y_out, T_out, status, n_substeps,
                          n_newton, scratch, cuda_stream, nullptr);
}

int kt_integrate_rad(const kt_network *net, int64_t ncells, const double *y_in, const double *T_in,
                     const double *rho, const double *flux, const double *path, double dt,
                     const kt_options *opts, double *y_out, double *T_out, int32_t *status,
                     int32_t *n_substeps, int32_t *n_newton, void *scratch, void *cuda_stream)
{
    return integrate_impl(net, ncells, y_in, T_in, rho, nullptr, dt, opts, y_out, T_out, status, n_substeps,
                          n_newton, scratch, cuda_stream, nullptr, nullptr, flux, path);
}

int kt_integrate_dt(const kt_network *net, int64_t ncells, const double *y_in, const double *T_in,
                    const double *rho, const double *dt_cells, const kt_options *opts, double *y_out,
                    double *T_out, int32_t *status, int32_t *n_substeps, int32_t *n_newton, void *scratch,
                    void *cuda_stream)
{
    if (!dt_cells) return fail(KT_EINVAL, "kt_integrate_dt: NULL dt_cells");
    return integrate_impl(net, ncells, y_in, T_in, rho, dt_cells, 1.0, opts, y_out, T_out, status, n_substeps,
                          n_newton, scratch, cuda_stream, nullptr);
}

int kt_scratch_check(void *scratch, void *cuda_stream)
{
    if (!scratch) return fail(KT_EINVAL, "kt_scratch_check: NULL scratch");
    kt::Scratch h{};
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemcpyAsync(&h, scratch, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "kt_scratch_check");
    if (h.error != 0) {
        int zero = 0;
        cudaMemcpyAsync(reinterpret_cast<char *>(scratch) + offsetof(kt::Scratch, error), &zero, sizeof zero,
                        cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        return fail(KT_ETIMEOUT, "device: a bounded wait for the network-table copy gave up (code %d)", h.error);
    }
    return KT_OK;
}

int kt_state_create(const kt_network *net, int64_t ncells, kt_state **out)
{
    if (!net || !out || ncells < 0) return fail(KT_EINVAL, "kt_state_create: bad argument");
    *out = nullptr;
    kt_state *st = new (std::nothrow) kt_state();
    if (!st) return fail(KT_ENOMEM, "kt_state_create: out of memory");
    st->net = net;
    st->ncells = ncells;
    cudaGetDevice(&st->device);
    const size_t n = static_cast<size_t>(ncells > 0 ? ncells : 1);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc(reinterpret_cast<void **>(&st->y), n * net->ns * sizeof(double));
    alloc(reinterpret_cast<void **>(&st->T), n * sizeof(double));
    alloc(reinterpret_cast<void **>(&st->rho), n * sizeof(double));
    alloc(reinterpret_cast<void **>(&st->status), n * sizeof(int));
    alloc(reinterpret_cast<void **>(&st->nsub), n * sizeof(int));
    alloc(reinterpret_cast<void **>(&st->nnew), n * sizeof(int));
    alloc(reinterpret_cast<void **>(&st->scratch), sizeof(kt::Scratch));
    if (e == cudaSuccess) e = cudaMemset(st->scratch, 0, sizeof(kt::Scratch));
    if (e == cudaSuccess) e = cudaMemset(st->status, 0, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(st->nsub, 0, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(st->nnew, 0, n * sizeof(int));
    if (e != cudaSuccess) {
        kt_state_free(st);
        return fail(KT_ENOMEM, "kt_state_create: %s", cudaGetErrorString(e));
    }
    *out = st;
    return KT_OK;
}

void kt_state_free(kt_state *st)
{
    if (!st) return;
    if (st->mlp) kt_mlp_free(st->mlp);
    if (st->gexec) cudaGraphExecDestroy(st->gexec);
    if (st->cap) cudaStreamDestroy(st->cap);
    cudaFree(st->y);
    cudaFree(st->T);
    cudaFree(st->rho);
    cudaFree(st->status);
    cudaFree(st->nsub);
    cudaFree(st->nnew);
    cudaFree(st->scratch);
    cudaFree(st->order);
    cudaFree(st->sched_work);
    delete st;
}

int kt_state_upload(kt_state *st, const double *y, const double *T, const double *rho, int src_is_device,
                    void *cuda_stream)
{
    if (!st || !y || !T) return fail(KT_EINVAL, "kt_state_upload: NULL argument");
    if (st->ncells == 0) return KT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const cudaMemcpyKind k = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t n = static_cast<size_t>(st->ncells);
    cudaError_t e = cudaMemcpyAsync(st->y, y, n * st->net->ns * sizeof(double), k, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st->T, T, n * sizeof(double), k, s);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(st->rho, rho, n * sizeof(double), k, s);
    if (e == cudaSuccess && !rho) {
        // ordered on the caller's stream; a pageable source is staged before the call
        // returns, so the local vector may go out of scope
        std::vector<double> ones(n, 1.0);
        e = cudaMemcpyAsync(st->rho, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "kt_state_upload");
    return KT_OK;
}

int kt_state_set_cost(kt_state *st, const int32_t *cost, int src_is_device, void *cuda_stream)
{
    if (!st || !cost) return fail(KT_EINVAL, "kt_state_set_cost: NULL argument");
    if (st->ncells == 0) return KT_OK;
    const cudaMemcpyKind k = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(st->nnew, cost, static_cast<size_t>(st->ncells) * sizeof(int32_t), k,
                                    static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? KT_OK : cuda_fail(e, "kt_state_set_cost");
}

int kt_integrate(kt_state *st, double dt, const kt_options *opts, void *cuda_stream)
{
    if (!st) return fail(KT_EINVAL, "kt_integrate: NULL state");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!opts || !opts->use_graph || st->ncells == 0) {
        const int *order = nullptr;
        if (opts && st->ncells > 0) {
            int rc = check_opts(opts);
            if (rc) return rc;
            rc = state_schedule(st, opts, s, true, &order);
            if (rc) return rc;
        }
        return integrate_impl(st->net, st->ncells, st->y, st->T, st->rho, nullptr, dt, opts, st->y, st->T,
                              st->status, st->nsub, st->nnew, st->scratch, cuda_stream, st->mlp, order);
    }
    int rc = check_opts(opts);
    if (rc) return rc;
    if (st->gexec && st->g_dt == dt && std::memcmp(&st->g_opts, opts, sizeof(kt_options)) == 0) {
        cudaError_t e = cudaGraphLaunch(st->gexec, s);
        return e == cudaSuccess ? KT_OK : cuda_fail(e, "cudaGraphLaunch");
    }
    // upload the network tables and allocate the schedule buffers first: no
    // synchronous call may run inside the capture
    const unsigned char *blob = nullptr;
    rc = const_cast<kt_network *>(st->net)->device_blob(&blob);
    if (rc) return rc;
    const int *order = nullptr;
    rc = state_schedule(st, opts, s, false, &order);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (!st->cap) e = cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate(capture)");
    e = cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    rc = state_schedule(st, opts, st->cap, true, &order);
    if (!rc)
        rc = integrate_impl(st->net, st->ncells, st->y, st->T, st->rho, nullptr, dt, opts, st->y, st->T,
                            st->status, st->nsub, st->nnew, st->scratch, st->cap, st->mlp, order);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    if (st->gexec) {
        cudaGraphExecDestroy(st->gexec);
        st->gexec = nullptr;
    }
    e = cudaGraphInstantiate(&st->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    st->g_dt = dt;
    st->g_opts = *opts;
    e = cudaGraphLaunch(st->gexec, s);
    return e == cudaSuccess ? KT_OK : cuda_fail(e, "cudaGraphLaunch");
}

int kt_network_attach_mlp(kt_network *net, const kt_mlp *mlp)
{
    if (!net) return fail(KT_EINVAL, "kt_network_attach_mlp: NULL network");
    net->mlp = mlp;
    return KT_OK;
}

int kt_mlp_load(kt_state *st, const char *weights_path)
{
    if (!st || !weights_path) return fail(KT_EINVAL, "kt_mlp_load: NULL argument");
    kt_mlp *m = nullptr;
    int rc = kt_mlp_load_file(weights_path, &m);
    if (rc) return rc;
    if (st->mlp) kt_mlp_free(st->mlp);
    st->mlp = m;
    if (st->gexec) {
        cudaGraphExecDestroy(st->gexec);
        st->gexec = nullptr;
    }
    return KT_OK;
}

int kt_autotune(const kt_network *net, int64_t ncells, const double *y_in, const double *T_in, double dt,
                const kt_options *base, double *y_out, double *T_out, void *scratch, void *cuda_stream,
                kt_options *best, double *best_seconds)
{
    if (!net || !base || !best || ncells <= 0) return fail(KT_EINVAL, "kt_autotune: bad argument");
    int rc = check_opts(base);
    if (rc) return rc;
    const int N = net->ns + net->energy;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(e, "kt_autotune: cudaEventCreate");
    double best_t = 1e300;
    kt_options cand = *base, win = *base;
    // The kernel family follows the size unless the caller fixed it: one cell per lane
    // when it fits (every FP64 warp instruction then serves 32 cells), else one per
    // warp.  A short tuning sample cannot judge that choice (short integrations are
    // latency-bound and favour one cell per warp), so only the launch shape is searched.
    const int fam = base->cells_per_warp ? base->cells_per_warp : (N <= kt::kLaneMaxN ? 32 : 1);
    const int cpws[1] = {fam};
    const int bws[4] = {1, 2, 4, 8};
    // the FP32-LU lane kernels under TR-BDF2 come in two storage variants (kt.h KT_LANE_*)
    const bool two = fam == 32 && base->form == KT_FORM_FP32LU && base->scheme == KT_SCHEME_TRBDF2 &&
                     base->lane_variant == KT_LANE_AUTO;
    const int vars[2] = {two ? KT_LANE_JCACHE : base->lane_variant, KT_LANE_LEAN};
    for (int ci = 0; ci < 1; ++ci) {
        if (cpws[ci] == 32 && N > kt::kLaneMaxN) continue;
        for (int vi = 0; vi < (two ? 2 : 1); ++vi)
        for (int per = 0; per <= 1; ++per)
            for (int bi = 0; bi < 4; ++bi) {
                cand.cells_per_warp = cpws[ci];
                cand.lane_variant = vars[vi];
                cand.persistent = per;
                cand.block_warps = bws[bi];
                cand.blocks_per_sm = 0;
                cand.use_graph = 0;
                rc = kt_integrate_ptrs(net, ncells, y_in, T_in, nullptr, dt, &cand, y_out, T_out, nullptr, nullptr,
                                       nullptr, scratch, cuda_stream);
                if (rc) break;
                cudaEventRecord(e0, s);
                rc = kt_integrate_ptrs(net, ncells, y_in, T_in, nullptr, dt, &cand, y_out, T_out, nullptr, nullptr,
                                       nullptr, scratch, cuda_stream);
                cudaEventRecord(e1, s);
                if (rc) break;
                e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "kt_autotune: run");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_t) {
                    best_t = ms;
                    win = cand;
                }
            }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *best = win;
    if (best_seconds) *best_seconds = best_t * 1e-3;
    return KT_OK;
}

int kt_state_check(const kt_state *st, void *cuda_stream)
{
    if (!st) return fail(KT_EINVAL, "kt_state_check: NULL state");
    return kt_scratch_check(st->scratch, cuda_stream);
}

int kt_state_download(const kt_state *st, double *y, double *T, int32_t *status, int32_t *n_substeps,
                      int32_t *n_newton, int dst_is_device, void *cuda_stream)
{
    if (!st) return fail(KT_EINVAL, "kt_state_download: NULL state");
    if (st->ncells == 0) return KT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t n = static_cast<size_t>(st->ncells);
    cudaError_t e = cudaSuccess;
    if (y) e = cudaMemcpyAsync(y, st->y, n * st->net->ns * sizeof(double), k, s);
    if (e == cudaSuccess && T) e = cudaMemcpyAsync(T, st->T, n * sizeof(double), k, s);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, st->status, n * sizeof(int), k, s);
    if (e == cudaSuccess && n_substeps) e = cudaMemcpyAsync(n_substeps, st->nsub, n * sizeof(int), k, s);
    if (e == cudaSuccess && n_newton) e = cudaMemcpyAsync(n_newton, st->nnew, n * sizeof(int), k, s);
    if (e != cudaSuccess) return cuda_fail(e, "kt_state_download");
    if (!dst_is_device) return kt_scratch_check(st->scratch, cuda_stream);
    return KT_OK;
}

}  // extern "C"
