// Les Houches Event files (hep-ph/0609017; version 3.0 adds per-event weight
// blocks): the "parse events" and "return new weights" steps of the
// reweighting procedure (Sec. 3.2, steps 2 and 8), host-side.
//
// Reading: the file is loaded once and its <event> blocks indexed; events are
// parsed in parallel (std::thread, contiguous ranges) with locale-independent
// number conversion (std::from_chars).  Each event's first line is
//   NUP IDPRUP XWGTUP SCALUP AQEDUP AQCDUP
// followed by NUP particle lines
//   IDUP ISTUP MOTHUP1 MOTHUP2 ICOLUP1 ICOLUP2 PX PY PZ E M VTIMUP SPINUP.
// Incoming (ISTUP = -1) and outgoing (ISTUP = +1) particles are matched, in
// file order, to the library's particle order of the process by PDG code;
// intermediate lines (ISTUP = 2, ...) are skipped.  The momenta are boosted
// along the beam axis into the partonic centre-of-mass frame (the frame the
// kernels and the mass-shell reshuffle assume; |M|^2 itself is invariant) and
// stored as [N][4][ld] (E, px, py, pz); XWGTUP is the weight.
//
// Writing: the original text, with each event's new weights added as
//   <wgt id='ID'> value </wgt>
// lines inside its <rwgt> block (created before </event> when absent).
#include <algorithm>
#include <charconv>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <string_view>
#include <thread>
#include <vector>

#include "../../include/rwgt.h"

struct rw_lhe {
  std::string text;
  std::vector<size_t> body, end;  // per event: first byte after "<event...>", position of "</event>"
  std::string err;
  // streaming writer (rw_lhe_write_begin/events/end)
  FILE* wf = nullptr;
  size_t w_at = 0;        // text written up to here
  int64_t w_next = 0;     // next event to write
  std::vector<std::string> w_ids;
};

namespace {

int lhe_fail(rw_lhe* h, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int lhe_fail(rw_lhe* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return code;
}

// particle order of each process in the kernels (PDG codes)
bool process_codes(int process, std::vector<int>& codes) {
  switch (process) {
    case RW_EE_MUMU: codes = {11, -11, 13, -13}; return true;
    case RW_GG_TT: codes = {21, 21, 6, -6}; return true;
    case RW_GG_TTG: codes = {21, 21, 6, -6, 21}; return true;
    case RW_GG_TTGG: codes = {21, 21, 6, -6, 21, 21}; return true;
    case RW_EE_5A: codes = {11, -11, 22, 22, 22, 22, 22}; return true;
  }
  return false;
}

struct Cursor {
  const char* p;
  const char* e;
  void skip_ws() {
    while (p < e && (*p == ' ' || *p == '\t' || *p == '\r' || *p == '\n')) ++p;
  }
  // a real number; Fortran's D exponent (1.5D+02) is read as E
  bool num(double& v) {
    skip_ws();
    if (p < e && *p == '+') ++p;
    auto r = std::from_chars(p, e, v);
    if (r.ec != std::errc()) return false;
    if (r.ptr < e && (*r.ptr == 'D' || *r.ptr == 'd')) {
      char buf[64];
      const char* t = r.ptr + 1;
      while (t < e && ((*t >= '0' && *t <= '9') || ((*t == '+' || *t == '-') && t == r.ptr + 1))) ++t;
      const size_t n = (size_t)(t - p);
      if (t == r.ptr + 1 || n >= sizeof buf) return false;
      std::memcpy(buf, p, n);
      buf[r.ptr - p] = 'E';
      const auto r2 = std::from_chars(buf, buf + n, v);
      if (r2.ec != std::errc() || r2.ptr != buf + n) return false;
      p = t;
      return true;
    }
    p = r.ptr;
    return true;
  }
  bool num(long long& v) {
    skip_ws();
    if (p < e && *p == '+') ++p;
    auto r = std::from_chars(p, e, v);
    if (r.ec != std::errc()) return false;
    p = r.ptr;
    return true;
  }
};

struct Particle {
  long long id, status;
  double px, py, pz, e;
};

// parse event k into out[N][4] (E, px, py, pz) and its weight; 0 or an error index
int parse_event(const rw_lhe* h, size_t k, const std::vector<int>& codes, double (*out)[4], double& w,
                std::string& why) {
  Cursor c{h->text.data() + h->body[k], h->text.data() + h->end[k]};
  double d;
  long long nup, idprup;
  if (!c.num(nup) || !c.num(idprup) || !c.num(w) || !c.num(d) || !c.num(d) || !c.num(d)) {
    why = "bad event header line";
    return 1;
  }
  if (nup < 1 || nup > 64) {
    why = "NUP out of range";
    return 1;
  }
  Particle ps[64];
  for (long long i = 0; i < nup; ++i) {
    long long m1, m2, c1, c2;
    double mass, vt, sp;
    Particle& q = ps[i];
    if (!c.num(q.id) || !c.num(q.status) || !c.num(m1) || !c.num(m2) || !c.num(c1) || !c.num(c2) || !c.num(q.px) ||
        !c.num(q.py) || !c.num(q.pz) || !c.num(q.e) || !c.num(mass) || !c.num(vt) || !c.num(sp)) {
      why = "bad particle line";
      return 1;
    }
  }
  const int N = (int)codes.size();
  bool used[64] = {};
  for (int s = 0; s < N; ++s) {
    const long long want_status = s < 2 ? -1 : 1;
    int found = -1;
    for (long long i = 0; i < nup && found < 0; ++i)
      if (!used[i] && ps[i].status == want_status && ps[i].id == codes[s]) found = (int)i;
    if (found < 0) {
      why = "particles do not match the process";
      return 1;
    }
    used[found] = true;
    out[s][0] = ps[found].e;
    out[s][1] = ps[found].px;
    out[s][2] = ps[found].py;
    out[s][3] = ps[found].pz;
  }
  for (long long i = 0; i < nup; ++i)
    if (!used[i] && (ps[i].status == -1 || ps[i].status == 1)) {
      why = "extra external particles for the process";
      return 1;
    }
  // boost along z into the centre-of-mass frame of the two incoming partons
  const double et = out[0][0] + out[1][0], pzt = out[0][3] + out[1][3];
  if (!(et > 0.0) || !(std::fabs(pzt) < et)) {
    why = "unphysical incoming momenta";
    return 1;
  }
  if (pzt != 0.0) {
    const double b = pzt / et, g = 1.0 / std::sqrt((1.0 - b) * (1.0 + b));
    for (int s = 0; s < N; ++s) {
      const double e0 = out[s][0], z0 = out[s][3];
      out[s][0] = g * (e0 - b * z0);
      out[s][3] = g * (z0 - b * e0);
    }
  }
  return 0;
}

}  // namespace

extern "C" {

int rw_lhe_open(rw_lhe** out, const char* path) {
  if (!out || !path) return RW_ERR_NULL;
  *out = nullptr;
  rw_lhe* h = new rw_lhe();
  FILE* f = fopen(path, "rb");
  if (!f) {
    delete h;
    return RW_ERR_ARG;
  }
  fseek(f, 0, SEEK_END);
  const long sz = ftell(f);
  fseek(f, 0, SEEK_SET);
  h->text.resize(sz > 0 ? (size_t)sz : 0);
  const size_t got = sz > 0 ? fread(&h->text[0], 1, (size_t)sz, f) : 0;
  fclose(f);
  if (sz < 0 || got != (size_t)sz) {
    delete h;
    return RW_ERR_ARG;
  }
  // index the <event> blocks: after </init> when there is one, skipping XML
  // comments (a file may mention "<event>" or "</event>" in one).  Between
  // blocks the next "<event" is searched once and only the text before it is
  // searched for "<!--"; inside a block "</event>" and "<!--" are searched
  // from the current position on.  Every character is looked at a bounded
  // number of times, so the scan is linear in the file size.  A comment that
  // is never closed, or an <event> that is never closed, makes the file
  // unreadable (RW_ERR_ARG): indexing past it would silently drop events.
  const std::string& t = h->text;
  const std::string_view tv(t);
  const size_t npos = std::string::npos;
  const size_t init_end = t.find("</init>");
  size_t pos = init_end == npos ? 0 : init_end + 7;
  size_t ev = t.find("<event", pos);
  for (;;) {
    if (ev != npos && ev < pos) ev = t.find("<event", pos);
    const size_t lim = ev == npos ? t.size() : ev;
    const size_t cm = tv.substr(pos, lim - pos).find("<!--");
    if (cm != std::string_view::npos) {
      const size_t ce = t.find("-->", pos + cm + 4);
      if (ce == npos) {
        delete h;
        return RW_ERR_ARG;
      }
      pos = ce + 3;
      continue;
    }
    if (ev == npos) break;
    pos = ev;
    const char nx = pos + 6 < t.size() ? t[pos + 6] : '\0';
    if (nx != '>' && nx != ' ' && nx != '\t' && nx != '\n' && nx != '\r') {  // e.g. <eventgroup>
      pos += 6;
      continue;
    }
    const size_t gt = t.find('>', pos);
    // the block ends at the first "</event>" outside a comment
    size_t close = npos, ce = npos;
    for (size_t q = gt == npos ? npos : gt + 1; q != npos;) {
      if (ce == npos || ce < q) ce = t.find("</event>", q);
      if (ce == npos) break;
      const size_t c0 = tv.substr(q, ce - q).find("<!--");
      if (c0 == std::string_view::npos) {
        close = ce;
        break;
      }
      const size_t c1 = t.find("-->", q + c0 + 4);
      q = c1 == npos ? npos : c1 + 3;
    }
    if (close == npos) {
      delete h;
      return RW_ERR_ARG;
    }
    h->body.push_back(gt + 1);
    h->end.push_back(close);
    pos = close + 8;
  }
  *out = h;
  return RW_OK;
}

int rw_lhe_close(rw_lhe* h) {
  if (!h) return RW_ERR_NULL;
  if (h->wf) fclose(h->wf);
  delete h;
  return RW_OK;
}

const char* rw_lhe_last_error(const rw_lhe* h) { return h ? h->err.c_str() : "null handle"; }

int64_t rw_lhe_n_events(const rw_lhe* h) { return h ? (int64_t)h->body.size() : -1; }

}  // extern "C"

namespace {

// parse the events idx(0..n-1) into columns 0..n-1 of h_mom [N][4][ld] and
// h_w with up to n_threads threads (contiguous shares of the list)
template <class Index>
int read_events(rw_lhe* h, int process, int64_t n, Index idx, double* h_mom, int64_t ld, double* h_w,
                int n_threads) {
  std::vector<int> codes;
  if (!process_codes(process, codes)) return lhe_fail(h, RW_ERR_ARG, "unknown process %d", process);
  const int N = (int)codes.size();
  const int T = std::max(1, std::min<int>(n_threads > 0 ? n_threads : 1, (int)std::max<int64_t>(1, n / 1024)));
  std::vector<long long> bad(T, -1);
  std::vector<std::string> why(T);
  auto work = [&](int t) {
    const int64_t a = n * t / T, b = n * (t + 1) / T;
    double p[16][4];
    for (int64_t i = a; i < b; ++i) {
      double w;
      const int64_t k = idx(i);
      if (parse_event(h, (size_t)k, codes, p, w, why[t])) {
        bad[t] = k;
        return;
      }
      for (int s = 0; s < N; ++s)
        for (int m = 0; m < 4; ++m) h_mom[((int64_t)s * 4 + m) * ld + i] = p[s][m];
      h_w[i] = w;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
  for (int t = 0; t < T; ++t)
    if (bad[t] >= 0) return lhe_fail(h, RW_ERR_ARG, "event %lld: %s", bad[t], why[t].c_str());
  return RW_OK;
}

}  // namespace

extern "C" {

int rw_lhe_read(rw_lhe* h, int process, int64_t first, int64_t n, double* h_mom, int64_t ld, double* h_w,
                int n_threads) {
  if (!h) return RW_ERR_NULL;
  if (!h_mom || !h_w) return lhe_fail(h, RW_ERR_NULL, "momenta/weights are NULL");
  if (first < 0 || n < 0 || first + n > (int64_t)h->body.size() || ld < n)
    return lhe_fail(h, RW_ERR_ARG, "range [%lld, %lld) / ld %lld outside the %zu events", (long long)first,
                    (long long)(first + n), (long long)ld, h->body.size());
  return read_events(h, process, n, [first](int64_t i) { return first + i; }, h_mom, ld, h_w, n_threads);
}

int rw_lhe_read_list(rw_lhe* h, int process, const int64_t* idx, int64_t n, double* h_mom, int64_t ld, double* h_w,
                     int n_threads) {
  if (!h) return RW_ERR_NULL;
  if (!h_mom || !h_w || (n > 0 && !idx)) return lhe_fail(h, RW_ERR_NULL, "index list, momenta or weights are NULL");
  if (n < 0 || ld < n) return lhe_fail(h, RW_ERR_ARG, "n %lld / ld %lld", (long long)n, (long long)ld);
  const int64_t E = (int64_t)h->body.size();
  for (int64_t i = 0; i < n; ++i)
    if (idx[i] < 0 || idx[i] >= E)
      return lhe_fail(h, RW_ERR_ARG, "index %lld: event %lld outside the %lld events", (long long)i,
                      (long long)idx[i], (long long)E);
  return read_events(h, process, n, [idx](int64_t i) { return idx[i]; }, h_mom, ld, h_w, n_threads);
}

int rw_lhe_classify(rw_lhe* h, const int* processes, int n_processes, int* h_process_of_event, int n_threads) {
  if (!h) return RW_ERR_NULL;
  if (!processes || !h_process_of_event) return lhe_fail(h, RW_ERR_NULL, "process list or output is NULL");
  if (n_processes < 1 || n_processes > 8) return lhe_fail(h, RW_ERR_ARG, "1..8 processes");
  std::vector<std::vector<int>> codes(n_processes);
  for (int j = 0; j < n_processes; ++j)
    if (!process_codes(processes[j], codes[j])) return lhe_fail(h, RW_ERR_ARG, "unknown process %d", processes[j]);
  const int64_t E = (int64_t)h->body.size();
  const int T = std::max(1, std::min<int>(n_threads > 0 ? n_threads : 1, (int)std::max<int64_t>(1, E / 1024)));
  auto work = [&](int t) {
    double p[16][4], w;
    std::string why;
    for (int64_t k = E * t / T; k < E * (t + 1) / T; ++k) {
      int found = -1;
      for (int j = 0; j < n_processes && found < 0; ++j)
        if (!parse_event(h, (size_t)k, codes[j], p, w, why)) found = processes[j];
      h_process_of_event[k] = found;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
  return RW_OK;
}

int rw_lhe_write_begin(rw_lhe* h, const char* path, int P, const char* const* ids) {
  if (!h) return RW_ERR_NULL;
  if (!path || !ids) return lhe_fail(h, RW_ERR_NULL, "path and ids are required");
  if (h->wf) return lhe_fail(h, RW_ERR_STATE, "a write is already open");
  if (P < 1) return lhe_fail(h, RW_ERR_ARG, "need P >= 1");
  for (int j = 0; j < P; ++j) {
    if (!ids[j] || !*ids[j]) return lhe_fail(h, RW_ERR_ARG, "id %d is empty", j);
    for (const char* q = ids[j]; *q; ++q)
      if (*q == '\'' || *q == '<' || *q == '>' || *q == '&') return lhe_fail(h, RW_ERR_ARG, "id %d: bad character", j);
  }
  h->wf = fopen(path, "wb");
  if (!h->wf) return lhe_fail(h, RW_ERR_ARG, "cannot open %s", path);
  h->w_ids.assign(ids, ids + P);
  h->w_at = 0;
  h->w_next = 0;
  return RW_OK;
}

int rw_lhe_write_events(rw_lhe* h, int64_t first, int64_t n, const double* h_wnew, int64_t ld) {
  if (!h) return RW_ERR_NULL;
  if (!h->wf) return lhe_fail(h, RW_ERR_STATE, "no write open");
  if (!h_wnew && n > 0) return lhe_fail(h, RW_ERR_NULL, "weights are NULL");
  const int64_t E = (int64_t)h->body.size();
  if (first != h->w_next || n < 0 || first + n > E || ld < n)
    return lhe_fail(h, RW_ERR_ARG, "events [%lld, %lld) with ld %lld: next expected %lld of %lld", (long long)first,
                    (long long)(first + n), (long long)ld, (long long)h->w_next, (long long)E);
  const std::string& t = h->text;
  const int P = (int)h->w_ids.size();
  // per event: where the weight lines go and whether an <rwgt> block exists
  // (searched within the event's own block only: linear in the file size)
  std::vector<size_t> cut(n);
  std::vector<char> has(n);
  const std::string_view tv(t);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t k = first + i;
    const std::string_view blk = tv.substr(h->body[k], h->end[k] - h->body[k]);
    const size_t rb = blk.find("<rwgt>");
    has[i] = rb != std::string_view::npos;
    const size_t re = has[i] ? blk.find("</rwgt>", rb) : blk.size();
    if (re == std::string_view::npos)
      return lhe_fail(h, RW_ERR_ARG, "event %lld: unclosed <rwgt>", (long long)k);
    cut[i] = h->body[k] + re;
  }
  // the inserted text of every event, formatted in parallel: the shortest
  // decimal form that reads back as the same double (std::to_chars)
  const int T = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), (int)(n / 4096) + 1));
  std::vector<std::string> ins(n);
  auto fmt = [&](int th) {
    char num[64];
    for (int64_t i = n * th / T; i < n * (th + 1) / T; ++i) {
      std::string& o = ins[i];
      if (!has[i]) o += "<rwgt>\n";
      for (int j = 0; j < P; ++j) {
        auto r = std::to_chars(num, num + sizeof num, h_wnew[(int64_t)j * ld + i]);
        o += "<wgt id='";
        o += h->w_ids[j];
        o += "'> ";
        o.append(num, r.ptr);
        o += " </wgt>\n";
      }
      if (!has[i]) o += "</rwgt>\n";
    }
  };
  {
    std::vector<std::thread> pool;
    for (int th = 1; th < T; ++th) pool.emplace_back(fmt, th);
    fmt(0);
    for (auto& x : pool) x.join();
  }
  bool ok = true;
  for (int64_t i = 0; i < n && ok; ++i) {
    ok = fwrite(t.data() + h->w_at, 1, cut[i] - h->w_at, h->wf) == cut[i] - h->w_at &&
         fwrite(ins[i].data(), 1, ins[i].size(), h->wf) == ins[i].size();
    h->w_at = cut[i];
  }
  if (!ok) return lhe_fail(h, RW_ERR_ARG, "write failed");
  h->w_next = first + n;
  return RW_OK;
}

int rw_lhe_write_end(rw_lhe* h) {
  if (!h) return RW_ERR_NULL;
  if (!h->wf) return lhe_fail(h, RW_ERR_STATE, "no write open");
  const int64_t E = (int64_t)h->body.size();
  const std::string& t = h->text;
  bool ok = h->w_next == E;
  if (ok) ok = fwrite(t.data() + h->w_at, 1, t.size() - h->w_at, h->wf) == t.size() - h->w_at;
  if (fclose(h->wf) != 0) ok = false;
  h->wf = nullptr;
  if (h->w_next != E)
    return lhe_fail(h, RW_ERR_STATE, "only %lld of %lld events written", (long long)h->w_next, (long long)E);
  return ok ? RW_OK : lhe_fail(h, RW_ERR_ARG, "write failed");
}

int rw_lhe_write(rw_lhe* h, const char* path, const double* h_wnew, int P, int64_t ld, const char* const* ids) {
  if (!h) return RW_ERR_NULL;
  if (!path || !h_wnew || !ids) return lhe_fail(h, RW_ERR_NULL, "path, weights and ids are required");
  const int64_t E = (int64_t)h->body.size();
  if (P < 1 || ld < E) return lhe_fail(h, RW_ERR_ARG, "need P >= 1 and ld >= %lld", (long long)E);
  int rc = rw_lhe_write_begin(h, path, P, ids);
  if (rc) return rc;
  rc = rw_lhe_write_events(h, 0, E, h_wnew, ld);
  const int rc2 = rw_lhe_write_end(h);
  return rc ? rc : rc2;
}

}  // extern "C"
