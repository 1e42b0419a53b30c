// Command-line front end of the GSGP library, after the paper's tool
// (Sec. 5, "How to use"): run parameters in a config file, training and
// test cases in text files (one case per row, features then the target in
// the last column), and as output, per generation, the training RMSE of the
// best individual and the test RMSE of the same individual.  Beyond the
// paper's tool it writes each run's best model (ancestor program plus one
// coefficient per random tree) to a text file, and applies such a file to
// new cases.
//
//   gsgp -train_file train.txt -test_file test.txt [-config config.ini]
//        [-output_dir DIR] [-batch]
//   gsgp -model DIR/model_run0.txt -predict_file cases.txt [-output y.txt]
//
// Config keys (key = value, '#' or ';' comments, [sections] ignored): the
// fields of gsgp_config (seed, run, pop_size, n_random_trees, pop_min_depth,
// pop_max_depth, rt_min_depth, rt_max_depth, const_lo, const_hi,
// p_grow_function, p_feature_given_terminal, protect_eps, ms, ms_mode,
// tournament_size, elitism, sigma_dtype, init_mode, max_genes, p_crossover)
// plus generations and runs.  Run k uses Philox counter word run + k.  Runs
// with crossover (p_crossover > 0) write no model file: their best
// individual is not an ancestor plus coefficients.
#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "gsgp.h"

namespace {

struct Dataset {
  std::vector<float> X;   // row-major n x l
  std::vector<float> y;
  int64_t n = 0;
  int l = 0;
};

[[noreturn]] void die(const std::string &msg) {
  fprintf(stderr, "gsgp: %s\n", msg.c_str());
  exit(2);
}

std::string trim(const std::string &s) {
  const size_t a = s.find_first_not_of(" \t\r\n");
  if (a == std::string::npos) return "";
  const size_t b = s.find_last_not_of(" \t\r\n");
  return s.substr(a, b - a + 1);
}

// Cases: rows of numbers separated by spaces, tabs or commas; the last
// column is the target.  Blank lines and lines starting with '#' are skipped.
Dataset read_cases(const std::string &path, bool with_target, int expect_features) {
  std::ifstream in(path);
  if (!in) die("cannot open " + path);
  Dataset d;
  std::string line;
  int64_t row = 0;
  int cols = -1;
  std::vector<float> vals;
  while (std::getline(in, line)) {
    ++row;
    const std::string t = trim(line);
    if (t.empty() || t[0] == '#') continue;
    vals.clear();
    const char *p = t.c_str();
    while (*p) {
      while (*p == ' ' || *p == '\t' || *p == ',') ++p;
      if (!*p) break;
      char *end = nullptr;
      errno = 0;
      const double v = strtod(p, &end);
      if (end == p || errno == ERANGE || !std::isfinite(v))
        die(path + ":" + std::to_string(row) + ": not a finite number");
      vals.push_back((float)v);
      p = end;
    }
    if (cols < 0) cols = (int)vals.size();
    if ((int)vals.size() != cols)
      die(path + ":" + std::to_string(row) + ": " + std::to_string(vals.size()) +
          " columns, expected " + std::to_string(cols));
    const int nf = with_target ? cols - 1 : cols;
    if (nf < 1) die(path + ": needs at least one feature column" +
                    std::string(with_target ? " and the target" : ""));
    d.X.insert(d.X.end(), vals.begin(), vals.begin() + nf);
    if (with_target) d.y.push_back(vals[(size_t)nf]);
    d.l = nf;
    ++d.n;
  }
  if (d.n == 0) die(path + ": no cases");
  if (expect_features > 0 && d.l != expect_features)
    die(path + ": " + std::to_string(d.l) + " features, expected " +
        std::to_string(expect_features));
  return d;
}

struct Settings {
  gsgp_config cfg;
  int generations = 100;
  int runs = 1;
};

Settings read_config(const std::string &path) {
  Settings s;
  gsgp_config_default(&s.cfg);
  if (path.empty()) return s;
  std::ifstream in(path);
  if (!in) die("cannot open " + path);
  std::string line;
  int row = 0;
  while (std::getline(in, line)) {
    ++row;
    std::string t = trim(line);
    const size_t c = t.find_first_of("#;");
    if (c != std::string::npos) t = trim(t.substr(0, c));
    if (t.empty() || t[0] == '[') continue;
    const size_t eq = t.find('=');
    if (eq == std::string::npos) die(path + ":" + std::to_string(row) + ": expected key = value");
    const std::string key = trim(t.substr(0, eq)), val = trim(t.substr(eq + 1));
    char *end = nullptr;
    const double v = strtod(val.c_str(), &end);
    if (val.empty() || *end != '\0')
      die(path + ":" + std::to_string(row) + ": " + key + " needs a number");
    gsgp_config &f = s.cfg;
    const std::map<std::string, int32_t *> ints = {
        {"pop_size", &f.pop_size}, {"n_random_trees", &f.n_random_trees},
        {"pop_min_depth", &f.pop_min_depth}, {"pop_max_depth", &f.pop_max_depth},
        {"rt_min_depth", &f.rt_min_depth}, {"rt_max_depth", &f.rt_max_depth},
        {"ms_mode", &f.ms_mode}, {"tournament_size", &f.tournament_size},
        {"elitism", &f.elitism}, {"sigma_dtype", &f.sigma_dtype}, {"init_mode", &f.init_mode},
        {"max_genes", &f.max_genes}};
    const std::map<std::string, float *> floats = {
        {"const_lo", &f.const_lo}, {"const_hi", &f.const_hi},
        {"p_grow_function", &f.p_grow_function},
        {"p_feature_given_terminal", &f.p_feature_given_terminal},
        {"protect_eps", &f.protect_eps}, {"ms", &f.ms}, {"p_crossover", &f.p_crossover}};
    if (ints.count(key)) {
      *ints.at(key) = (int32_t)v;
    } else if (floats.count(key)) {
      *floats.at(key) = (float)v;
    } else if (key == "seed") {
      f.seed = (uint64_t)v;
    } else if (key == "run") {
      f.run = (uint32_t)v;
    } else if (key == "generations") {
      s.generations = (int)v;
    } else if (key == "runs") {
      s.runs = (int)v;
    } else {
      die(path + ":" + std::to_string(row) + ": unknown key " + key);
    }
  }
  if (s.generations < 0) die("generations must be >= 0");
  if (s.runs < 1 || s.runs > 1024) die("runs must be in [1, 1024]");
  const char *bad = gsgp_config_error(&s.cfg);
  if (bad && *bad) die(path + ": " + bad);
  return s;
}

// ---- model files ---------------------------------------------------------
// Text, one item per line: header, fields, the ancestor program, then one
// line per random tree with a nonzero coefficient: coefficient, length and
// (gene, constant) pairs.  Floats are written in hexadecimal so that a model
// file reproduces the model bit for bit.
struct Model {
  int n_features = 0, sigma_dtype = 0, init_mode = 0;
  float protect_eps = 1e-3f;
  double best_train = 0, best_test = 0;
  std::vector<int> anc_genes;
  std::vector<float> anc_consts;
  std::vector<double> coef;
  std::vector<std::vector<int>> rt_genes;
  std::vector<std::vector<float>> rt_consts;
};

void write_program(FILE *f, const int *g, const float *c, int len) {
  fprintf(f, " %d", len);
  for (int k = 0; k < len; ++k) fprintf(f, " %d %a", g[k], (double)c[k]);
  fprintf(f, "\n");
}

void save_model(const std::string &path, const gsgp_trace &t, const std::vector<int> &tg,
                const std::vector<float> &tc) {
  FILE *f = fopen(path.c_str(), "w");
  if (!f) die("cannot write " + path);
  fprintf(f, "gsgp-model 1\n");
  fprintf(f, "n_features %d\nsigma_dtype %d\ninit_mode %d\nprotect_eps %a\n", t.n_features,
          t.sigma_dtype, t.init_mode, (double)t.protect_eps);
  fprintf(f, "best_train_rmse %a\nbest_test_rmse %a\n", t.best_train_rmse, t.best_test_rmse);
  fprintf(f, "ancestor");
  write_program(f, t.ancestor_genes, t.ancestor_consts, t.ancestor_length);
  int nk = 0;
  for (int k = 0; k < t.n_random_trees; ++k) nk += t.coef[k] != 0.0;
  fprintf(f, "terms %d\n", nk);
  for (int k = 0; k < t.n_random_trees; ++k) {
    if (t.coef[k] == 0.0) continue;
    fprintf(f, "%a", t.coef[k]);
    write_program(f, &tg[(size_t)k * t.rt_max_genes], &tc[(size_t)k * t.rt_max_genes],
                  t.rt_lengths[k]);
  }
  if (fclose(f) != 0) die("cannot write " + path);
}

Model load_model(const std::string &path) {
  std::ifstream in(path);
  if (!in) die("cannot open " + path);
  Model m;
  std::string word, line;
  auto expect = [&](const char *w) {
    if (!(in >> word) || word != w) die(path + ": expected " + std::string(w));
  };
  auto read_program = [&](std::vector<int> &g, std::vector<float> &c) {
    int len = -1;
    if (!(in >> len) || len < 0 || len > 65536) die(path + ": bad program length");
    g.resize((size_t)len);
    c.resize((size_t)len);
    for (int k = 0; k < len; ++k) {
      std::string cs;
      if (!(in >> g[(size_t)k] >> cs)) die(path + ": truncated program");
      c[(size_t)k] = (float)strtod(cs.c_str(), nullptr);
    }
  };
  auto read_hex = [&](double &v) {
    std::string s;
    if (!(in >> s)) die(path + ": truncated");
    v = strtod(s.c_str(), nullptr);
  };
  int version = 0;
  expect("gsgp-model");
  if (!(in >> version) || version != 1) die(path + ": unsupported model version");
  double pe = 0;
  expect("n_features");
  in >> m.n_features;
  expect("sigma_dtype");
  in >> m.sigma_dtype;
  expect("init_mode");
  in >> m.init_mode;
  expect("protect_eps");
  read_hex(pe);
  m.protect_eps = (float)pe;
  expect("best_train_rmse");
  read_hex(m.best_train);
  expect("best_test_rmse");
  read_hex(m.best_test);
  expect("ancestor");
  read_program(m.anc_genes, m.anc_consts);
  int nk = 0;
  expect("terms");
  if (!(in >> nk) || nk < 0 || nk > 65536) die(path + ": bad term count");
  m.coef.resize((size_t)nk);
  m.rt_genes.resize((size_t)nk);
  m.rt_consts.resize((size_t)nk);
  for (int q = 0; q < nk; ++q) {
    read_hex(m.coef[(size_t)q]);
    read_program(m.rt_genes[(size_t)q], m.rt_consts[(size_t)q]);
  }
  if (!in) die(path + ": truncated model");
  return m;
}

void check(gsgp_status st, gsgp_ctx *c, const char *what) {
  if (st != GSGP_OK) die(std::string(what) + ": " + (c ? gsgp_last_error(c) : "failed"));
}

int run_mode(const std::string &train, const std::string &test, const std::string &config,
             const std::string &outdir, bool batched) {
  Settings s = read_config(config);
  const Dataset tr = read_cases(train, true, 0);
  Dataset te;
  if (!test.empty()) te = read_cases(test, true, tr.l);
  const int G = s.generations, R = s.runs;
  std::vector<gsgp_ctx *> runs((size_t)R, nullptr);
  for (int k = 0; k < R; ++k) {
    gsgp_config cfg = s.cfg;
    cfg.run = s.cfg.run + (uint32_t)k;
    check(gsgp_create(&cfg, &runs[(size_t)k]), nullptr, "gsgp_create");
    gsgp_ctx *c = runs[(size_t)k];
    check(gsgp_load(c, tr.X.data(), tr.y.data(), tr.n, tr.l, te.n ? te.X.data() : nullptr,
                    te.n ? te.y.data() : nullptr, te.n),
          c, "gsgp_load");
    check(gsgp_init(c), c, "gsgp_init");
  }
  std::vector<double> btr((size_t)R * G), bte((size_t)R * G);
  if (batched && R > 1) {
    gsgp_batch *b = nullptr;
    if (gsgp_batch_create(runs.data(), R, &b) != GSGP_OK) die("gsgp_batch_create failed");
    if (G > 0 && gsgp_batch_evolve(b, G, btr.data(), bte.data()) != GSGP_OK)
      die(std::string("gsgp_batch_evolve: ") + gsgp_batch_last_error(b));
    gsgp_batch_destroy(b);
  } else {
    for (int k = 0; k < R; ++k)
      if (G > 0)
        check(gsgp_evolve(runs[(size_t)k], G, &btr[(size_t)k * G], &bte[(size_t)k * G]),
              runs[(size_t)k], "gsgp_evolve");
  }
  // per generation: one line, one column per run
  const std::string ftr = outdir + "/fitness_train.txt", fte = outdir + "/fitness_test.txt";
  FILE *a = fopen(ftr.c_str(), "w"), *b = fopen(fte.c_str(), "w");
  if (!a || !b) die("cannot write the fitness files in " + outdir);
  for (int g = 0; g < G; ++g) {
    for (int k = 0; k < R; ++k) {
      fprintf(a, k ? " %.17g" : "%.17g", btr[(size_t)k * G + g]);
      fprintf(b, k ? " %.17g" : "%.17g", bte[(size_t)k * G + g]);
    }
    fprintf(a, "\n");
    fprintf(b, "\n");
  }
  fclose(a);
  fclose(b);
  for (int k = 0; k < R; ++k) {
    gsgp_ctx *c = runs[(size_t)k];
    if (s.cfg.p_crossover > 0.0f) {
      if (G > 0)
        printf("run %d: best training RMSE %.9g, test RMSE %.9g\n", k,
               btr[(size_t)k * G + G - 1], bte[(size_t)k * G + G - 1]);
      gsgp_destroy(c);
      continue;
    }
    gsgp_trace t{};
    t.struct_size = sizeof t;
    check(gsgp_best_trace(c, &t), c, "gsgp_best_trace");   // sizes
    std::vector<int> ag((size_t)t.max_genes), rg((size_t)t.n_random_trees * t.rt_max_genes),
        rl((size_t)t.n_random_trees);
    std::vector<float> ac((size_t)t.max_genes), rc(rg.size());
    std::vector<double> coef((size_t)t.n_random_trees);
    t.ancestor_genes = ag.data();
    t.ancestor_consts = ac.data();
    t.coef = coef.data();
    t.rt_genes = rg.data();
    t.rt_consts = rc.data();
    t.rt_lengths = rl.data();
    check(gsgp_best_trace(c, &t), c, "gsgp_best_trace");
    save_model(outdir + "/model_run" + std::to_string(k) + ".txt", t, rg, rc);
    printf("run %d: best training RMSE %.9g, test RMSE %.9g\n", k, t.best_train_rmse,
           t.best_test_rmse);
    gsgp_destroy(c);
  }
  return 0;
}

int predict_mode(const std::string &model_path, const std::string &cases,
                 const std::string &output) {
  const Model m = load_model(model_path);
  const Dataset d = read_cases(cases, false, m.n_features);
  const int nk = (int)m.coef.size();
  int Kr = 1;
  for (const auto &g : m.rt_genes) Kr = g.size() > (size_t)Kr ? (int)g.size() : Kr;
  std::vector<int> rg((size_t)(nk ? nk : 1) * Kr, -1), rl((size_t)(nk ? nk : 1), 0);
  std::vector<float> rc(rg.size(), 0.0f);
  for (int q = 0; q < nk; ++q) {
    std::copy(m.rt_genes[(size_t)q].begin(), m.rt_genes[(size_t)q].end(), &rg[(size_t)q * Kr]);
    std::copy(m.rt_consts[(size_t)q].begin(), m.rt_consts[(size_t)q].end(), &rc[(size_t)q * Kr]);
    rl[(size_t)q] = (int)m.rt_genes[(size_t)q].size();
  }
  std::vector<int> ag = m.anc_genes;
  std::vector<float> ac = m.anc_consts;
  if (ag.empty()) {
    ag.push_back(-1);
    ac.push_back(0.0f);
  }
  std::vector<double> coef = m.coef;
  gsgp_trace t{};
  t.struct_size = sizeof t;
  t.ancestor_length = (int)m.anc_genes.size();
  t.max_genes = (int)ag.size();
  t.ancestor_genes = ag.data();
  t.ancestor_consts = ac.data();
  t.n_random_trees = nk;
  t.coef = coef.data();
  t.rt_max_genes = Kr;
  t.rt_genes = rg.data();
  t.rt_consts = rc.data();
  t.rt_lengths = rl.data();
  t.sigma_dtype = m.sigma_dtype;
  t.n_features = m.n_features;
  t.protect_eps = m.protect_eps;
  t.init_mode = m.init_mode;
  std::vector<double> y((size_t)d.n);
  char err[256];
  if (gsgp_model_predict(&t, d.X.data(), d.n, y.data(), nullptr, err, sizeof err) != GSGP_OK)
    die(std::string("gsgp_model_predict: ") + err);
  FILE *f = output.empty() ? stdout : fopen(output.c_str(), "w");
  if (!f) die("cannot write " + output);
  for (double v : y) fprintf(f, "%.17g\n", v);
  if (f != stdout) fclose(f);
  return 0;
}

void usage() {
  fprintf(stderr,
          "usage: gsgp -train_file FILE [-test_file FILE] [-config FILE] [-output_dir DIR] "
          "[-batch]\n"
          "       gsgp -model FILE -predict_file FILE [-output FILE]\n");
}

}  // namespace

int main(int argc, char **argv) {
  std::map<std::string, std::string> opt;
  bool batched = false;
  for (int k = 1; k < argc; ++k) {
    const std::string a = argv[k];
    if (a == "-batch") {
      batched = true;
    } else if (a == "-h" || a == "-help" || a == "--help") {
      usage();
      return 0;
    } else if ((a == "-train_file" || a == "-test_file" || a == "-config" || a == "-output_dir" ||
                a == "-model" || a == "-predict_file" || a == "-output") && k + 1 < argc) {
      opt[a] = argv[++k];
    } else {
      usage();
      die("unknown or incomplete option " + a);
    }
  }
  if (opt.count("-model")) {
    if (!opt.count("-predict_file")) die("-model needs -predict_file");
    return predict_mode(opt["-model"], opt["-predict_file"], opt["-output"]);
  }
  if (!opt.count("-train_file")) {
    usage();
    die("missing -train_file");
  }
  const std::string outdir = opt.count("-output_dir") ? opt["-output_dir"] : ".";
  return run_mode(opt["-train_file"], opt["-test_file"], opt["-config"], outdir, batched);
}
