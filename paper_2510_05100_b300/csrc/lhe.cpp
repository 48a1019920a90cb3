// LHE v3 front-end of the reweighting path (host code).
//
// Paper Sec. 2: events are read from an LHE file, sorted into processes by
// comparing their external legs (eventBelongs), reindexed to the process's
// parton order and transposed to a structure of arrays, the layout the
// reweighting kernels take.  Sec. 3.1: the new weights are appended to every
// event (<rwgt><wgt id=...>) and declared in the header's <initrwgt> block.
//
// Reading: the whole file is loaded, the <event> spans are found by one scan,
// then the events are parsed in parallel (std::thread, contiguous ranges) into
// flat particle arrays (PDG code, status, E px py pz, SPINUP) with std::from_chars.
// Writing: the original text is copied with the weight lines and the
// <initrwgt> group inserted (events formatted in parallel, written in order);
// nothing else changes.
#include <algorithm>
#include <charconv>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <string_view>
#include <thread>
#include <vector>

#include "../../include/rex.h"

namespace {

thread_local std::string g_lerr;
int lfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_lerr = buf;
  return code;
}

struct Event {
  int64_t start = 0, end = 0;   // text span of <event ...> ... </event>
  int64_t first = 0;            // index of its first particle
  int nup = 0;
  double xwgt = 0.0;
};

bool is_space(char c) { return c == ' ' || c == '\t' || c == '\r'; }

// Parsing cursor over one event's text; numbers are separated by blanks.
struct Cursor {
  const char* p;
  const char* end;
  bool ok = true;
  void skip_blank_lines() {
    while (p < end && (is_space(*p) || *p == '\n')) ++p;
  }
  template <typename T>
  T num() {
    while (p < end && is_space(*p)) ++p;
    if (p < end && *p == '+') ++p;
    T v{};
    const auto r = std::from_chars(p, end, v);
    if (r.ec != std::errc()) {
      ok = false;
      return T{};
    }
    p = r.ptr;
    return v;
  }
  // true when only blanks remain before the end of the line
  bool at_eol() {
    while (p < end && is_space(*p)) ++p;
    return p >= end || *p == '\n';
  }
  void next_line() {
    while (p < end && *p != '\n') ++p;
    if (p < end) ++p;
  }
};

// <tag followed by '>' or blank: the position, or npos
size_t find_tag(const std::string& s, const char* tag, size_t from) {
  const size_t n = std::strlen(tag);
  for (size_t pos = s.find(tag, from); pos != std::string::npos; pos = s.find(tag, pos + 1)) {
    const char c = pos + n < s.size() ? s[pos + n] : '\0';
    if (c == '>' || is_space(c) || c == '\n') return pos;
  }
  return std::string::npos;
}

}  // namespace

struct rex_lhe {
  std::string text;
  size_t init_at = 0;
  std::vector<Event> ev;
  std::vector<int> pdg, status;
  std::vector<double> mom;   // [particles][4] E, px, py, pz
  std::vector<signed char> spin;   // SPINUP rounded to an integer; 9 (unknown) when absent
  std::vector<std::string> wid;
  std::vector<std::vector<double>> wval;   // [id][event], NaN where unset
  std::vector<std::vector<char>> whas;
};

extern "C" {

const char* rex_lhe_last_error(void) { return g_lerr.c_str(); }

int rex_lhe_read(const char* path, int nthreads, rex_lhe** out) {
  if (!out || !path) return lfail(REX_EINVAL, "null argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return lfail(REX_EINVAL, "cannot open %s", path);
  rex_lhe* L = new (std::nothrow) rex_lhe();
  if (!L) {
    std::fclose(f);
    return lfail(REX_ENOMEM, "out of host memory");
  }
  std::fseek(f, 0, SEEK_END);
  const long size = std::ftell(f);
  std::fseek(f, 0, SEEK_SET);
  L->text.resize(size > 0 ? (size_t)size : 0);
  const size_t got = size > 0 ? std::fread(&L->text[0], 1, (size_t)size, f) : 0;
  std::fclose(f);
  if ((long)got != size) {
    delete L;
    return lfail(REX_EINVAL, "short read of %s", path);
  }
  const std::string& s = L->text;
  L->init_at = find_tag(s, "<init", 0);
  if (L->init_at == std::string::npos) {
    delete L;
    return lfail(REX_EINVAL, "%s: no <init> block", path);
  }
  // event spans
  for (size_t pos = find_tag(s, "<event", L->init_at); pos != std::string::npos;) {
    const size_t close = s.find("</event>", pos);
    if (close == std::string::npos) {
      delete L;
      return lfail(REX_EINVAL, "%s: unterminated event at byte %zu", path, pos);
    }
    Event e;
    e.start = (int64_t)pos;
    e.end = (int64_t)(close + 8);
    L->ev.push_back(e);
    pos = find_tag(s, "<event", close + 8);
  }
  const int64_t nev = (int64_t)L->ev.size();
  int nt = nthreads > 0 ? nthreads : (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > 256) nt = 256;
  if (nev < 4096) nt = 1;
  auto for_ranges = [&](auto&& body) {
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) {
      const int64_t a = nev * t / nt, b = nev * (t + 1) / nt;
      th.emplace_back([&body, a, b]() { body(a, b); });
    }
    for (auto& x : th) x.join();
  };
  // pass 1: the first line of every event (nUP, xWgtUP)
  std::vector<char> bad(nev, 0);
  for_ranges([&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      Event& e = L->ev[i];
      Cursor c{s.data() + s.find('>', e.start) + 1, s.data() + e.end};
      c.skip_blank_lines();
      e.nup = c.num<int>();
      c.num<int>();
      e.xwgt = c.num<double>();
      if (!c.ok || e.nup < 0 || e.nup > 1000) bad[i] = 1;
    }
  });
  for (int64_t i = 0; i < nev; ++i)
    if (bad[i]) {
      delete L;
      return lfail(REX_EINVAL, "%s: malformed first line in event %lld", path, (long long)i);
    }
  int64_t np = 0;
  for (auto& e : L->ev) {
    e.first = np;
    np += e.nup;
  }
  L->pdg.resize(np);
  L->status.resize(np);
  L->mom.resize((size_t)np * 4);
  L->spin.resize(np);
  // pass 2: the particle lines
  for_ranges([&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      const Event& e = L->ev[i];
      Cursor c{s.data() + s.find('>', e.start) + 1, s.data() + e.end};
      c.skip_blank_lines();
      c.next_line();
      for (int k = 0; k < e.nup; ++k) {
        c.skip_blank_lines();
        const int64_t q = e.first + k;
        L->pdg[q] = c.num<int>();
        L->status[q] = c.num<int>();
        for (int u = 0; u < 4; ++u) c.num<int>();   // mothers, colours
        const double px = c.num<double>(), py = c.num<double>(), pz = c.num<double>(), en = c.num<double>();
        double* m = &L->mom[(size_t)q * 4];
        m[0] = en;
        m[1] = px;
        m[2] = py;
        m[3] = pz;
        // m, VTIMUP, SPINUP: optional trailing columns (SPINUP 9 = unknown when absent)
        double sp = 9.0;
        if (!c.at_eol()) {
          c.num<double>();
          if (!c.at_eol()) {
            c.num<double>();
            if (!c.at_eol()) sp = c.num<double>();
          }
        }
        const double r = std::nearbyint(sp);
        L->spin[q] = !(r == r) ? (signed char)9 : (signed char)(r > 127.0 ? 127 : (r < -127.0 ? -127 : r));
        c.next_line();
      }
      if (!c.ok) bad[i] = 1;
    }
  });
  for (int64_t i = 0; i < nev; ++i)
    if (bad[i]) {
      delete L;
      return lfail(REX_EINVAL, "%s: malformed particle line in event %lld", path, (long long)i);
    }
  *out = L;
  return REX_OK;
}

int64_t rex_lhe_num_events(const rex_lhe* L) { return L ? (int64_t)L->ev.size() : REX_EINVAL; }

}  // extern "C"

// The events of one process (rex_lhe_extract, rex_lhe_extract_helicities): each
// output is optional; rows follow the file order, particles the requested order.
static int extract_impl(const rex_lhe* L, const int* pdg_in, int n_in, const int* pdg_out, int n_out, int64_t* nev,
                        double* momenta, double* weights, int64_t* index, signed char* helicities) {
  if (!L || !nev || n_in < 0 || n_out < 0 || n_in + n_out < 1 || n_in + n_out > 64 ||
      (n_in && !pdg_in) || (n_out && !pdg_out))
    return lfail(REX_EINVAL, "bad arguments");
  std::vector<int> want_in(pdg_in, pdg_in + n_in), want_out(pdg_out, pdg_out + n_out);
  std::vector<int> sin = want_in, sout = want_out;
  std::sort(sin.begin(), sin.end());
  std::sort(sout.begin(), sout.end());
  const int npart = n_in + n_out;
  int64_t n = 0;
  std::vector<int> ci, co;
  std::vector<int64_t> qi, qo;
  std::vector<char> used;
  for (int64_t i = 0; i < (int64_t)L->ev.size(); ++i) {
    const Event& e = L->ev[i];
    ci.clear();
    co.clear();
    qi.clear();
    qo.clear();
    for (int k = 0; k < e.nup; ++k) {
      const int64_t q = e.first + k;
      if (L->status[q] == -1) {
        ci.push_back(L->pdg[q]);
        qi.push_back(q);
      } else if (L->status[q] == 1) {
        co.push_back(L->pdg[q]);
        qo.push_back(q);
      }
    }
    if ((int)ci.size() != n_in || (int)co.size() != n_out) continue;
    std::vector<int> a = ci, b = co;
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != sin || b != sout) continue;
    if (momenta) {
      double* row = momenta + (size_t)n * npart * 4;
      int slot = 0;
      for (int side = 0; side < 2; ++side) {
        const std::vector<int>& want = side ? want_out : want_in;
        const std::vector<int>& codes = side ? co : ci;
        const std::vector<int64_t>& qs = side ? qo : qi;
        used.assign(codes.size(), 0);
        for (int code : want) {
          size_t k = 0;
          while (used[k] || codes[k] != code) ++k;   // exists: the multisets match
          used[k] = 1;
          std::memcpy(row + 4 * slot, &L->mom[(size_t)qs[k] * 4], 4 * sizeof(double));
          ++slot;
        }
      }
    }
    if (helicities) {
      signed char* row = helicities + (size_t)n * npart;
      int slot = 0;
      for (int side = 0; side < 2; ++side) {
        const std::vector<int>& want = side ? want_out : want_in;
        const std::vector<int>& codes = side ? co : ci;
        const std::vector<int64_t>& qs = side ? qo : qi;
        used.assign(codes.size(), 0);
        for (int code : want) {
          size_t k = 0;
          while (used[k] || codes[k] != code) ++k;
          used[k] = 1;
          row[slot++] = L->spin[(size_t)qs[k]];
        }
      }
    }
    if (weights) weights[n] = e.xwgt;
    if (index) index[n] = i;
    ++n;
  }
  *nev = n;
  return REX_OK;
}

extern "C" {

int rex_lhe_extract(const rex_lhe* L, const int* pdg_in, int n_in, const int* pdg_out, int n_out, int64_t* nev,
                    double* momenta, double* weights, int64_t* index) {
  return extract_impl(L, pdg_in, n_in, pdg_out, n_out, nev, momenta, weights, index, nullptr);
}

int rex_lhe_extract_helicities(const rex_lhe* L, const int* pdg_in, int n_in, const int* pdg_out, int n_out,
                               int64_t* nev, signed char* helicities) {
  return extract_impl(L, pdg_in, n_in, pdg_out, n_out, nev, nullptr, nullptr, nullptr, helicities);
}

int rex_lhe_set_weights(rex_lhe* L, const char* id, const int64_t* index, const double* values, int64_t n) {
  if (!L || !id || (n > 0 && (!index || !values)) || n < 0) return lfail(REX_EINVAL, "bad arguments");
  if (!*id || std::strpbrk(id, "'<>&\"")) return lfail(REX_EINVAL, "weight id must be non-empty plain text");
  const int64_t nev = (int64_t)L->ev.size();
  for (int64_t i = 0; i < n; ++i)
    if (index[i] < 0 || index[i] >= nev) return lfail(REX_EINVAL, "event index %lld out of range", (long long)index[i]);
  size_t w = 0;
  while (w < L->wid.size() && L->wid[w] != id) ++w;
  if (w == L->wid.size()) {
    L->wid.emplace_back(id);
    L->wval.emplace_back(nev, NAN);
    L->whas.emplace_back(nev, 0);
  }
  for (int64_t i = 0; i < n; ++i) {
    L->wval[w][index[i]] = values[i];
    L->whas[w][index[i]] = 1;
  }
  return REX_OK;
}

// One event's text with its weight lines inserted, appended to out.
static void emit_event(const rex_lhe* L, size_t i, std::string& out, std::string& lines) {
  const std::string& s = L->text;
  const Event& e = L->ev[i];
  char buf[64];
  lines.clear();
  for (size_t w = 0; w < L->wid.size(); ++w)
    if (L->whas[w][i]) {
      // " %+.10e " with std::to_chars (correctly rounded, as printf)
      const double v = L->wval[w][i];
      char* p = buf;
      *p++ = ' ';
      if (!std::signbit(v)) *p++ = '+';
      p = std::to_chars(p, buf + sizeof buf - 2, v, std::chars_format::scientific, 10).ptr;
      *p++ = ' ';
      lines += "<wgt id='";
      lines += L->wid[w];
      lines += "'>";
      lines.append(buf, (size_t)(p - buf));
      lines += "</wgt>\n";
    }
  if (lines.empty()) {
    out.append(s, (size_t)e.start, (size_t)(e.end - e.start));
    return;
  }
  const size_t close = (size_t)e.end - 8;   // "</event>"
  // the event's last </rwgt>, searched inside the event only
  const std::string_view body(s.data() + e.start, close - (size_t)e.start);
  const size_t rb = body.rfind("</rwgt>");
  if (rb != std::string_view::npos) {
    const size_t r = (size_t)e.start + rb;
    out.append(s, (size_t)e.start, r - (size_t)e.start);
    out += lines;
    out.append(s, r, (size_t)e.end - r);
  } else {
    out.append(s, (size_t)e.start, close - (size_t)e.start);
    out += "<rwgt>\n";
    out += lines;
    out += "</rwgt>\n";
    out.append(s, close, 8);
  }
}

int rex_lhe_write(const rex_lhe* L, const char* path) {
  if (!L || !path) return lfail(REX_EINVAL, "null argument");
  const std::string& s = L->text;
  std::string header = s.substr(0, L->init_at);
  if (!L->wid.empty()) {
    std::string group = "<weightgroup name='rex_b300'>\n";
    for (const auto& id : L->wid) group += "<weight id='" + id + "'>" + id + "</weight>\n";
    group += "</weightgroup>\n";
    size_t k;
    if ((k = header.find("</initrwgt>")) != std::string::npos)
      header.insert(k, group);
    else if ((k = header.find("</header>")) != std::string::npos)
      header.insert(k, "<initrwgt>\n" + group + "</initrwgt>\n");
    else
      header += "<header>\n<initrwgt>\n" + group + "</initrwgt>\n</header>\n";
  }
  // events formatted in parallel, one text chunk per contiguous range (each range
  // also carries the original text between its events), written in order
  const int64_t nev = (int64_t)L->ev.size();
  int nt = (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > 64) nt = 64;
  if (nev < 4096) nt = 1;
  std::vector<std::string> chunk(nt);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    const int64_t a = nev * t / nt, b = nev * (t + 1) / nt;
    th.emplace_back([&, a, b, t]() {
      std::string& out = chunk[t];
      std::string lines;
      if (b > a) out.reserve((size_t)(L->ev[b - 1].end - L->ev[a].start) + (size_t)(b - a) * (16 + 48 * L->wid.size()));
      for (int64_t i = a; i < b; ++i) {
        // the text between the previous event (or the <init> block) and this one
        const size_t prev = i == 0 ? L->init_at : (size_t)L->ev[i - 1].end;
        out.append(s, prev, (size_t)L->ev[i].start - prev);
        emit_event(L, (size_t)i, out, lines);
      }
    });
  }
  for (auto& x : th) x.join();
  const size_t tail = nev ? (size_t)L->ev[nev - 1].end : L->init_at;
  FILE* f = std::fopen(path, "wb");
  if (!f) return lfail(REX_EINVAL, "cannot open %s for writing", path);
  bool ok = std::fwrite(header.data(), 1, header.size(), f) == header.size();
  for (const auto& c : chunk) ok = ok && std::fwrite(c.data(), 1, c.size(), f) == c.size();
  ok = ok && std::fwrite(s.data() + tail, 1, s.size() - tail, f) == s.size() - tail;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? REX_OK : lfail(REX_EINVAL, "short write to %s", path);
}

void rex_lhe_free(rex_lhe* L) { delete L; }

}  // extern "C"
