// jit.cu -- runtime generator: a tensor-index program -> CUDA source -> NVRTC -> one fused sm_103a kernel.
//
// The GB300 counterpart of the paper's CodeWriter (Secs. 3-4): instead of registering every expression
// template at link time and emitting one kernel per expression with one thread per (point, component),
// a whole program of index statements is parsed at run time and emitted as ONE kernel with one thread
// per grid point that evaluates every component of every statement, keeping intermediates (`temp`
// tensors) in registers and storing only the `out` tensors.
//
// Language (one declaration or statement per ';'):
//   in  NAME(d0, d1, ...) [sym(a,b) ...];   input tensor, slot dimensions (3 or 4), symmetric slot pairs
//   out NAME(...) [sym(...)];                output tensor        temp NAME(...) [sym(...)];  register-only
//   in  NAME;                                scalar (rank 0)
//   index l(d), m(d) ...;                    explicit ranges of index letters (default: the slot dimension)
//   NAME(idx, ...) = EXPR;                   statement; idx: letter, letter+k / letter-k (offset), integer
//   EXPR: numbers, NAME(idx...), + - * /, unary -, ( ), Sum(letter, EXPR)
// Index rules (the paper's, Sec. 2.3): both operands of + and - carry the same free indices; a letter
// may not appear in both factors of a product (contractions are written with Sum); the right-hand
// side's free indices equal the left-hand side's letters.  A letter ranges over its slot's dimension
// unless declared with `index l(d);` (the paper's spatial i_ on a spacetime slot).  Each stored
// component the left-hand side reaches is evaluated once, at the first index assignment (row-major)
// that reaches it -- a symmetric pair is stored once, as in the paper's lookup table.
// Component storage order of a tensor: its stored index tuples in row-major order.
#include "../../include/tl_testing.h"
#include <dlfcn.h>

#include <functional>

#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "tl_host.h"

namespace tl {
namespace jit {

// ---------------------------------------------------------------------------------------------- model
struct Tensor {
    std::string name;
    int kind = 0;                               // 0 in, 1 out, 2 temp
    std::vector<int> dims;
    std::vector<std::pair<int, int>> sym;       // symmetric slot pairs
    std::vector<std::vector<int>> stored;       // stored index tuples, storage order
    std::map<std::vector<int>, int> slot_of;    // any index tuple -> storage position
    int table_base = 0;                         // first position in the in/out table
};

struct Idx {
    bool fixed = false;
    int value = 0;      // fixed value, or offset
    char letter = 0;
};

struct Expr {
    enum Kind { NUM, REF, NEG, ADD, SUB, MUL, DIV, SUM } kind;
    double num = 0;
    int tensor = -1;
    std::vector<Idx> idx;
    char sum_letter = 0;
    std::unique_ptr<Expr> a, b;
};

struct Stmt {
    int tensor;
    std::vector<Idx> lhs;
    std::unique_ptr<Expr> rhs;
};

struct Program {
    std::map<char, int> ranges;                 // declared index ranges ("index i(3);")
    std::vector<Tensor> tensors;
    std::vector<Stmt> stmts;
    int n_in = 0, n_out = 0;
    std::string source, names;
    std::vector<uint8_t> reads;                 // per input table entry: does the kernel load it
};

struct Error {
    std::string msg;
};

// ----------------------------------------------------------------------------------------------- lexer
struct Lexer {
    const std::string &s;
    size_t p = 0;
    explicit Lexer(const std::string &src) : s(src) {}
    void ws()
    {
        while (p < s.size()) {
            if (isspace((unsigned char)s[p]))
                ++p;
            else if (s[p] == '#' || (s[p] == '/' && p + 1 < s.size() && s[p + 1] == '/'))
                while (p < s.size() && s[p] != '\n')
                    ++p;
            else
                break;
        }
    }
    bool eof()
    {
        ws();
        return p >= s.size();
    }
    char peek()
    {
        ws();
        return p < s.size() ? s[p] : '\0';
    }
    bool accept(char c)
    {
        if (peek() == c) {
            ++p;
            return true;
        }
        return false;
    }
    void expect(char c)
    {
        if (!accept(c))
            throw Error{std::string("expected '") + c + "' at offset " + std::to_string(p)};
    }
    std::string ident()
    {
        ws();
        size_t b = p;
        if (p < s.size() && (isalpha((unsigned char)s[p]) || s[p] == '_'))
            while (p < s.size() && (isalnum((unsigned char)s[p]) || s[p] == '_'))
                ++p;
        if (b == p)
            throw Error{"expected a name at offset " + std::to_string(p)};
        return s.substr(b, p - b);
    }
    bool at_number()
    {
        char c = peek();
        return isdigit((unsigned char)c) || c == '.';
    }
    double number()
    {
        ws();
        const char *b = s.c_str() + p;
        char *e = nullptr;
        double v = strtod(b, &e);
        if (e == b)
            throw Error{"expected a number at offset " + std::to_string(p)};
        p += (size_t)(e - b);
        return v;
    }
    int integer()
    {
        ws();
        size_t b = p;
        while (p < s.size() && isdigit((unsigned char)s[p]))
            ++p;
        if (b == p)
            throw Error{"expected an integer at offset " + std::to_string(p)};
        return atoi(s.substr(b, p - b).c_str());
    }
};

// ---------------------------------------------------------------------------------------------- parser
struct Parser {
    Lexer L;
    Program &P;
    std::map<std::string, int> by_name;
    Parser(const std::string &src, Program &prog) : L(src), P(prog) {}

    int tensor_id(const std::string &n)
    {
        auto it = by_name.find(n);
        if (it == by_name.end())
            throw Error{"unknown tensor '" + n + "'"};
        return it->second;
    }

    std::vector<Idx> index_list()
    {
        std::vector<Idx> v;
        if (!L.accept('('))
            return v;
        if (L.accept(')'))
            return v;
        do {
            Idx i;
            if (L.at_number()) {
                i.fixed = true;
                i.value = L.integer();
            } else {
                std::string id = L.ident();
                if (id.size() != 1 || !islower((unsigned char)id[0]))
                    throw Error{"index names are single lower-case letters (got '" + id + "')"};
                i.letter = id[0];
                if (L.accept('+'))
                    i.value = L.integer();
                else if (L.accept('-'))
                    i.value = -L.integer();
            }
            v.push_back(i);
        } while (L.accept(','));
        L.expect(')');
        return v;
    }

    void declaration(int kind)
    {
        Tensor t;
        t.kind = kind;
        t.name = L.ident();
        if (by_name.count(t.name))
            throw Error{"tensor '" + t.name + "' declared twice"};
        if (L.accept('(')) {
            if (!L.accept(')')) {
                do {
                    int d = L.integer();
                    if (d < 1 || d > 4)
                        throw Error{"slot dimension of '" + t.name + "' must be 1..4"};
                    t.dims.push_back(d);
                } while (L.accept(','));
                L.expect(')');
            }
        }
        while (!L.eof() && L.peek() != ';') {
            std::string kw = L.ident();
            if (kw != "sym")
                throw Error{"unexpected '" + kw + "' in the declaration of '" + t.name + "'"};
            L.expect('(');
            int a = L.integer();
            L.expect(',');
            int b = L.integer();
            L.expect(')');
            if (a == b || a < 0 || b < 0 || a >= (int)t.dims.size() || b >= (int)t.dims.size() || t.dims[a] != t.dims[b])
                throw Error{"bad sym(" + std::to_string(a) + "," + std::to_string(b) + ") for '" + t.name + "'"};
            t.sym.push_back({std::min(a, b), std::max(a, b)});
        }
        // stored components: canonical tuples (each symmetric pair ascending), row-major order
        const int rank = (int)t.dims.size();
        std::vector<int> tup(rank, 0);
        for (;;) {
            std::vector<int> canon = tup;
            bool changed = true;   // bubble through the pairs until every pair is ascending
            while (changed) {
                changed = false;
                for (auto &pr : t.sym)
                    if (canon[pr.first] > canon[pr.second]) {
                        std::swap(canon[pr.first], canon[pr.second]);
                        changed = true;
                    }
            }
            if (canon == tup) {
                t.slot_of[tup] = (int)t.stored.size();
                t.stored.push_back(tup);
            }
            int r = rank - 1;
            while (r >= 0 && ++tup[r] == t.dims[r])
                tup[r--] = 0;
            if (r < 0)
                break;
        }
        // every tuple maps to its canonical tuple's slot
        std::vector<int> all(rank, 0);
        for (;;) {
            std::vector<int> canon = all;
            bool changed = true;
            while (changed) {
                changed = false;
                for (auto &pr : t.sym)
                    if (canon[pr.first] > canon[pr.second]) {
                        std::swap(canon[pr.first], canon[pr.second]);
                        changed = true;
                    }
            }
            t.slot_of[all] = t.slot_of.at(canon);
            int r = rank - 1;
            while (r >= 0 && ++all[r] == t.dims[r])
                all[r--] = 0;
            if (r < 0)
                break;
        }
        by_name[t.name] = (int)P.tensors.size();
        P.tensors.push_back(std::move(t));
    }

    std::unique_ptr<Expr> primary()
    {
        auto e = std::make_unique<Expr>();
        if (L.accept('(')) {
            auto inner = sum_expr();
            L.expect(')');
            return inner;
        }
        if (L.accept('-')) {
            e->kind = Expr::NEG;
            e->a = primary();
            return e;
        }
        if (L.at_number()) {
            e->kind = Expr::NUM;
            e->num = L.number();
            return e;
        }
        std::string id = L.ident();
        if (id == "Sum") {
            L.expect('(');
            std::string l = L.ident();
            if (l.size() != 1 || !islower((unsigned char)l[0]))
                throw Error{"Sum needs a single-letter index"};
            L.expect(',');
            e->kind = Expr::SUM;
            e->sum_letter = l[0];
            e->a = sum_expr();
            L.expect(')');
            return e;
        }
        e->kind = Expr::REF;
        e->tensor = tensor_id(id);
        e->idx = index_list();
        if (e->idx.size() != P.tensors[e->tensor].dims.size())
            throw Error{"'" + id + "' has rank " + std::to_string(P.tensors[e->tensor].dims.size())};
        return e;
    }

    std::unique_ptr<Expr> product()
    {
        auto e = primary();
        for (;;) {
            Expr::Kind k;
            if (L.accept('*'))
                k = Expr::MUL;
            else if (L.accept('/'))
                k = Expr::DIV;
            else
                return e;
            auto n = std::make_unique<Expr>();
            n->kind = k;
            n->a = std::move(e);
            n->b = primary();
            e = std::move(n);
        }
    }

    std::unique_ptr<Expr> sum_expr()
    {
        auto e = product();
        for (;;) {
            Expr::Kind k;
            if (L.accept('+'))
                k = Expr::ADD;
            else if (L.accept('-'))
                k = Expr::SUB;
            else
                return e;
            auto n = std::make_unique<Expr>();
            n->kind = k;
            n->a = std::move(e);
            n->b = product();
            e = std::move(n);
        }
    }

    void parse()
    {
        while (!L.eof()) {
            size_t save = L.p;
            std::string id = L.ident();
            if (id == "index") {
                do {
                    std::string l = L.ident();
                    if (l.size() != 1 || !islower((unsigned char)l[0]))
                        throw Error{"index names are single lower-case letters (got '" + l + "')"};
                    L.expect('(');
                    const int d = L.integer();
                    L.expect(')');
                    if (d < 1 || d > 4)
                        throw Error{"index range must be 1..4"};
                    P.ranges[l[0]] = d;
                } while (L.accept(','));
                L.expect(';');
                continue;
            }
            if (id == "in" || id == "out" || id == "temp") {
                // "in NAME..." is a declaration unless "in" is itself followed by '(' or '='
                char c = L.peek();
                if (c != '(' && c != '=') {
                    declaration(id == "in" ? 0 : id == "out" ? 1 : 2);
                    L.expect(';');
                    continue;
                }
            }
            L.p = save;
            Stmt st;
            st.tensor = tensor_id(L.ident());
            if (P.tensors[st.tensor].kind == 0)
                throw Error{"cannot assign to input '" + P.tensors[st.tensor].name + "'"};
            st.lhs = index_list();
            if (st.lhs.size() != P.tensors[st.tensor].dims.size())
                throw Error{"left-hand side '" + P.tensors[st.tensor].name + "' has the wrong rank"};
            L.expect('=');
            st.rhs = sum_expr();
            L.expect(';');
            P.stmts.push_back(std::move(st));
        }
    }
};

// ------------------------------------------------------------------------------- index checks, codegen
using Binding = std::map<char, int>;

// Free letters of an expression and the slot dimension each is used with; throws on rule violations.
// `summed` holds the letters bound by enclosing Sums: only those may repeat (within one tensor or across
// the two factors of a product), since the Sum is what contracts them.
int range_of(const Program &P, char letter, int slot_dim)
{
    auto it = P.ranges.find(letter);
    return it != P.ranges.end() ? it->second : slot_dim;
}

void free_letters(const Program &P, const Expr &e, std::map<char, int> &out, const std::set<char> &summed)
{
    auto merge = [&](const std::map<char, int> &f, const std::map<char, int> &g, bool product) {
        for (auto &kv : g) {
            auto it = f.find(kv.first);
            if (it != f.end()) {
                if (product && !summed.count(kv.first))
                    throw Error{std::string("index '") + kv.first + "' appears in both factors of a product (use Sum)"};
            }
        }
    };
    switch (e.kind) {
    case Expr::NUM:
        return;
    case Expr::REF: {
        const Tensor &t = P.tensors[e.tensor];
        for (size_t s = 0; s < e.idx.size(); ++s)
            if (!e.idx[s].fixed) {
                // a free letter takes its range from the left-hand side (or its declaration); uses on
                // slots of other dimensions are bounds-checked when the code is generated
                const int d = range_of(P, e.idx[s].letter, t.dims[s]);
                auto it = out.find(e.idx[s].letter);
                if (it != out.end() && !summed.count(e.idx[s].letter))
                    throw Error{std::string("index '") + e.idx[s].letter + "' repeated within '" + t.name +
                                "' (write contractions with Sum)"};
                out[e.idx[s].letter] = d;
            }
        return;
    }
    case Expr::NEG:
        free_letters(P, *e.a, out, summed);
        return;
    case Expr::ADD:
    case Expr::SUB: {
        std::map<char, int> fa, fb;
        free_letters(P, *e.a, fa, summed);
        free_letters(P, *e.b, fb, summed);
        std::set<char> sa, sb;
        for (auto &kv : fa)
            sa.insert(kv.first);
        for (auto &kv : fb)
            sb.insert(kv.first);
        if (sa != sb)
            throw Error{"the operands of + / - carry different free indices"};
        out.insert(fa.begin(), fa.end());
        return;
    }
    case Expr::MUL:
    case Expr::DIV: {
        std::map<char, int> fa, fb;
        free_letters(P, *e.a, fa, summed);
        free_letters(P, *e.b, fb, summed);
        if (e.kind == Expr::DIV && !fb.empty())
            throw Error{"only scalar expressions may divide"};
        merge(fa, fb, true);
        out.insert(fa.begin(), fa.end());
        out.insert(fb.begin(), fb.end());
        return;
    }
    case Expr::SUM: {
        if (summed.count(e.sum_letter))
            throw Error{std::string("nested Sums over the same index '") + e.sum_letter + "'"};
        std::set<char> inner = summed;
        inner.insert(e.sum_letter);
        std::map<char, int> fa;
        free_letters(P, *e.a, fa, inner);
        if (!fa.count(e.sum_letter))
            throw Error{std::string("Sum over '") + e.sum_letter + "', which is not free in its operand"};
        fa.erase(e.sum_letter);
        merge(out, fa, false);
        out.insert(fa.begin(), fa.end());
        return;
    }
    }
}

// The range of a summation letter inside e: its declaration, or the common dimension of the slots it
// indexes (an error when they differ and no declaration settles it).
int letter_dim(const Program &P, const Expr &e, char l)
{
    std::set<int> dims;
    std::function<void(const Expr &)> walk = [&](const Expr &x) {
        if (x.kind == Expr::REF) {
            for (size_t s = 0; s < x.idx.size(); ++s)
                if (!x.idx[s].fixed && x.idx[s].letter == l)
                    dims.insert(range_of(P, l, P.tensors[x.tensor].dims[s]));
        }
        if (x.a)
            walk(*x.a);
        if (x.b)
            walk(*x.b);
    };
    walk(e);
    if (dims.size() != 1)
        throw Error{std::string("summation index '") + l + "' indexes slots of different dimensions: declare its range"};
    return *dims.begin();
}

std::string value_name(const Program &P, int tensor, int slot)
{
    const Tensor &t = P.tensors[tensor];
    return (t.kind == 0 ? "in_" : "v_") + t.name + "_" + std::to_string(slot);
}

std::string fmt_num(double v)
{
    char b[64];
    snprintf(b, sizeof b, "%.17g", v);
    std::string s(b);
    if (s.find_first_of(".eEn") == std::string::npos)
        s += ".0";
    return "(" + s + ")";
}

// Code generation state for one kernel: inputs read, components defined so far, hoisted reciprocals.
struct GenState {
    std::set<int> used_inputs;
    std::vector<std::set<int>> defined;
    std::map<std::string, std::string> recip;   // divisor code -> variable holding its reciprocal
    std::map<std::string, std::string> scaled;  // "factor|k" -> variable holding factor * 2^k
    int hoisted = 0;                            // names of hoisted values are never reused
    std::ostringstream *body = nullptr;
};

std::string gen(const Program &P, const Expr &e, Binding &bind, GenState &G);

// One addend of a flattened sum: its sign, its code, and for a genuine product x * y (not an exact
// power-of-two scaling) the two factors, so that the sum can fuse it into an FMA.
struct Term {
    int sign;
    std::string code, x, y;
    bool prod;
};

// A genuine product (x * y, or x times a hoisted reciprocal): its factors' code; false for anything
// else, including a constant factor +-2^k, which becomes an exact exponent adjustment.
std::string factor_code(const Program &P, const Expr &f, Binding &bind, GenState &G);

bool product_factors(const Program &P, const Expr &e, Binding &bind, GenState &G, std::string &x, std::string &y)
{
    if (e.kind == Expr::DIV) {
        // divisors are scalars: one reciprocal per distinct divisor, computed where first needed
        const std::string den = gen(P, *e.b, bind, G);
        auto it = G.recip.find(den);
        if (it == G.recip.end()) {
            const std::string name = "r_" + std::to_string(G.hoisted++);
            *G.body << "    const double " << name << " = tl_rcp(" << den << ");\n";
            it = G.recip.emplace(den, name).first;
        }
        x = factor_code(P, *e.a, bind, G);
        y = it->second;
        return true;
    }
    if (e.kind != Expr::MUL)
        return false;
    for (int side = 0; side < 2; ++side) {
        const Expr &c = side ? *e.b : *e.a;
        const bool neg = c.kind == Expr::NEG && c.a->kind == Expr::NUM;
        const Expr &num = neg ? *c.a : c;
        if (num.kind == Expr::NUM && num.num != 0.0) {
            int k = 0;
            const double m = frexp(num.num, &k);   // num = m 2^k, m in [0.5, 1)
            if (m == 0.5 && k - 1 >= -8 && k - 1 <= 8 && k - 1 != 0)
                return false;
        }
    }
    x = factor_code(P, *e.a, bind, G);
    y = factor_code(P, *e.b, bind, G);
    return true;
}

// A factor of a product: a nested genuine product stays a plain FP64 multiply (the integer-pipe
// product is kept for the one product per sum that no FMA can absorb, which bounds the code size of
// programs such as Eqs. 17-20 whose terms are products of three or four factors).
std::string factor_code(const Program &P, const Expr &f, Binding &bind, GenState &G)
{
    std::string x, y;
    if (f.kind == Expr::MUL && product_factors(P, f, bind, G, x, y))
        return "(" + x + " * " + y + ")";
    return gen(P, f, bind, G);
}

// The addends of a chain of + / - / unary -, each with its sign, generated for the current binding.
void addends(const Program &P, const Expr &e, Binding &bind, GenState &G, int sign, std::vector<Term> &out)
{
    if (e.kind == Expr::ADD || e.kind == Expr::SUB) {
        addends(P, *e.a, bind, G, sign, out);
        addends(P, *e.b, bind, G, e.kind == Expr::ADD ? sign : -sign, out);
    } else if (e.kind == Expr::NEG) {
        addends(P, *e.a, bind, G, -sign, out);
    } else if (e.kind == Expr::SUM) {
        // a Sum of addends is itself a chain of additions
        const int d = letter_dim(P, *e.a, e.sum_letter);
        const bool shadow = bind.count(e.sum_letter) != 0;
        const int saved = shadow ? bind[e.sum_letter] : 0;
        for (int v = 0; v < d; ++v) {
            bind[e.sum_letter] = v;
            addends(P, *e.a, bind, G, sign, out);
        }
        if (shadow)
            bind[e.sum_letter] = saved;
        else
            bind.erase(e.sum_letter);
    } else {
        Term t{sign, "", "", "", false};
        t.prod = product_factors(P, e, bind, G, t.x, t.y);
        t.code = t.prod ? "tl_mul(" + t.x + ", " + t.y + ")" : gen(P, e, bind, G);
        out.push_back(t);
    }
}

// A signed sum.  Addends that are the same code with opposite signs cancel (e.g. the two bracket terms
// of Eq. 6 that name one stored element) and repeats merge into a coefficient.  The remaining plain
// addends are summed left to right, then those with a coefficient other than +-1 (a power of two fused
// into an FMA with the running sum: RN(s + 2^k a) in one operation, 2^k a being exact), then every
// product is fused into the running sum with an FMA, so a sum of products costs one stand-alone
// product (tl_mul, integer pipes) and FMAs.
std::string sum_code(const std::vector<Term> &terms)
{
    std::vector<Term> kept;
    for (auto &t : terms) {
        bool merged = false;
        for (auto &k : kept)
            if (k.code == t.code) {
                k.sign += t.sign;
                merged = true;
                break;
            }
        if (!merged)
            kept.push_back(t);
    }
    std::string s;
    for (int pass = 0; pass < 3; ++pass)
        for (auto &k : kept) {
            if (k.sign == 0)
                continue;
            const int mag = k.sign < 0 ? -k.sign : k.sign;
            const bool fuse = k.prod && mag == 1;
            const bool pow2 = (mag & (mag - 1)) == 0 && mag <= 256;
            const int want = fuse ? 2 : (mag > 1 && pow2 ? 1 : 0);
            if (want != pass)
                continue;
            if (fuse && !s.empty()) {
                s = "fma(" + (k.sign < 0 ? "(-" + k.x + ")" : k.x) + ", " + k.y + ", " + s + ")";
                continue;
            }
            if (pass == 1 && !s.empty()) {
                s = "fma(" + std::string(k.sign < 0 ? "-" : "") + std::to_string(mag) + ".0, " + k.code + ", " + s + ")";
                continue;
            }
            int lg = 0;
            while ((1 << lg) < mag)
                ++lg;
            const std::string term = mag == 1 ? k.code
                                     : pow2   ? "tl_pow2(" + k.code + ", " + std::to_string(lg) + ")"
                                              : "(" + std::to_string(mag) + ".0 * " + k.code + ")";
            if (s.empty())
                s = k.sign < 0 ? "(-" + term + ")" : term;
            else
                s = "(" + s + (k.sign < 0 ? " - " : " + ") + term + ")";
        }
    return s.empty() ? "(0.0)" : s;
}

std::string gen(const Program &P, const Expr &e, Binding &bind, GenState &G)
{
    switch (e.kind) {
    case Expr::NUM:
        return fmt_num(e.num);
    case Expr::REF: {
        const Tensor &t = P.tensors[e.tensor];
        std::vector<int> tup;
        for (size_t s = 0; s < e.idx.size(); ++s) {
            int v = e.idx[s].fixed ? e.idx[s].value : bind.at(e.idx[s].letter) + e.idx[s].value;
            if (v < 0 || v >= t.dims[s])
                throw Error{"index of '" + t.name + "' out of range (offset or fixed index)"};
            tup.push_back(v);
        }
        const int slot = t.slot_of.at(tup);
        if (t.kind == 0)
            G.used_inputs.insert(t.table_base + slot);
        else if (!G.defined[e.tensor].count(slot))
            throw Error{"component " + std::to_string(slot) + " of '" + t.name + "' is read before it is assigned"};
        return value_name(P, e.tensor, slot);
    }
    case Expr::NEG:
    case Expr::ADD:
    case Expr::SUB:
    case Expr::SUM: {
        std::vector<Term> terms;
        addends(P, e, bind, G, 1, terms);
        return sum_code(terms);
    }
    case Expr::MUL:
    case Expr::DIV: {
        std::string x, y;
        if (product_factors(P, e, bind, G, x, y))
            return "tl_mul(" + x + ", " + y + ")";
        // a constant factor +-2^k: an exact exponent adjustment on the integer pipe
        for (int side = 0; side < 2; ++side) {
            const Expr &c = side ? *e.b : *e.a;
            const Expr &other = side ? *e.a : *e.b;
            const bool neg = c.kind == Expr::NEG && c.a->kind == Expr::NUM;
            const Expr &num = neg ? *c.a : c;
            if (num.kind == Expr::NUM && num.num != 0.0) {
                int k = 0;
                const double m = frexp(num.num, &k);   // the side that product_factors found to be +-2^k
                if (m == 0.5 && k - 1 >= -8 && k - 1 <= 8 && k - 1 != 0) {
                    const std::string lg = std::to_string(k - 1);
                    // +-2^k times a sum whose addends are all genuine products: the scaling moves onto
                    // the first factor of each product (2^k a b = (2^k a) b exactly, away from the
                    // extremes of the range), where identical scaled factors are formed once, instead of
                    // onto every sum (the 1/2 of Eq. 6 on the 6 stored g^il rather than the 18 Gamma)
                    if (other.kind == Expr::ADD || other.kind == Expr::SUB || other.kind == Expr::NEG ||
                        other.kind == Expr::SUM) {
                        std::vector<Term> terms;
                        addends(P, other, bind, G, neg ? -1 : 1, terms);
                        bool all_prod = !terms.empty();
                        for (auto &t : terms)
                            all_prod = all_prod && t.prod;
                        if (all_prod) {
                            for (auto &t : terms) {
                                auto it = G.scaled.find(t.x + "|" + lg);
                                if (it == G.scaled.end()) {
                                    const std::string name = "s_" + std::to_string(G.hoisted++);
                                    *G.body << "    const double " << name << " = tl_pow2(" << t.x << ", " << lg << ");\n";
                                    it = G.scaled.emplace(t.x + "|" + lg, name).first;
                                }
                                t.x = it->second;
                                t.code = "tl_mul(" + t.x + ", " + t.y + ")";
                            }
                            return sum_code(terms);
                        }
                        return "tl_pow2(" + sum_code(terms) + ", " + lg + ")";
                    }
                    const std::string scaled = "tl_pow2(" + gen(P, other, bind, G) + ", " + lg + ")";
                    return neg ? "(-" + scaled + ")" : scaled;
                }
            }
        }
        return "";
    }
    }
    return "";
}

// The generated kernels' helpers.  Stand-alone binary64 product: the 106-bit product of the two 53-bit
// significands, normalised and rounded to nearest-even on the integer pipes, bit-identical to a * b;
// zero times finite gives the signed zero, other special or extreme operands take a * b out of line.
// (The same algorithm as the library kernels' product; NVRTC sees only this text.)
const char *const kMulSource =
    "__device__ __noinline__ double tl_mul_slow(double a, double b)\n{\n  return a * b;\n}\n"
    "__device__ __forceinline__ double tl_mul(double a, double b)\n{\n"
    "  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);\n"
    "  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);\n"
    "  const unsigned ea = (unsigned)(ua >> 52) & 0x7ffu, eb = (unsigned)(ub >> 52) & 0x7ffu;\n"
    "  const int e = (int)(ea + eb) - 1023;\n"
    "  const unsigned long long sign = (ua ^ ub) & 0x8000000000000000ull;\n"
    "  if (ea - 1u < 2046u && eb - 1u < 2046u && (unsigned)(e - 1) < 2044u) {\n"
    "    const unsigned long long ma = (ua & 0x000fffffffffffffull) | 0x0010000000000000ull;\n"
    "    const unsigned long long mb = (ub & 0x000fffffffffffffull) | 0x0010000000000000ull;\n"
    "    const unsigned long long lo = ma * mb, hi = __umul64hi(ma, mb);\n"
    "    const unsigned t = (unsigned)(hi >> 41);\n"
    "    const unsigned long long h = t ? hi : (hi << 1) | (lo >> 63), l = t ? lo : lo << 1;\n"
    "    unsigned long long m = (h << 11) | (l >> 53);\n"
    "    const unsigned long long rem = l & 0x001fffffffffffffull;\n"
    "    m += (rem + (m & 1ull) > 0x0010000000000000ull) ? 1ull : 0ull;\n"
    "    return __longlong_as_double((long long)(sign | (((unsigned long long)(e + (int)t - 1) << 52) + m)));\n"
    "  }\n"
    "  if (((ua << 1) == 0ull && eb != 0x7ffu) || ((ub << 1) == 0ull && ea != 0x7ffu))\n"
    "    return __longlong_as_double((long long)sign);\n"
    "  return tl_mul_slow(a, b);\n}\n"
    // reciprocal for the hoisted divisors: binary32 seed (rcp.approx on the bits of the binary32
    // truncation of d) and one third-order Newton-Raphson step e = 1 - d r, r' = r + r (e + e^2) in
    // binary64: relative error within one ulp for d inside the binary32 exponent range, 3 FMAs
    // instead of the division sequence; other d take 1.0 / d out of line
    "__device__ __noinline__ double tl_rcp_slow(double d)\n{\n  return 1.0 / d;\n}\n"
    "__device__ __forceinline__ double tl_rcp(double d)\n{\n"
    "  const unsigned long long b = (unsigned long long)__double_as_longlong(d);\n"
    "  const int e = (int)((b >> 52) & 0x7ff);\n"
    "  if (e > 1023 - 125 && e < 1023 + 125) {\n"
    "    const unsigned fb = (unsigned)((b >> 32) & 0x80000000u) | (unsigned)((e - 1023 + 127) << 23) |\n"
    "                        (unsigned)((b >> 29) & 0x7fffffu);\n"
    "    float rf;\n"
    "    asm(\"rcp.approx.ftz.f32 %0, %1;\" : \"=f\"(rf) : \"f\"(__uint_as_float(fb)));\n"
    "    const unsigned rb = __float_as_uint(rf);\n"
    "    const unsigned long long r64 = ((unsigned long long)(rb & 0x80000000u) << 32) |\n"
    "        ((unsigned long long)(((rb >> 23) & 0xff) - 127 + 1023) << 52) | ((unsigned long long)(rb & 0x7fffffu) << 29);\n"
    "    const double r = __longlong_as_double((long long)r64);\n"
    "    const double err = fma(-d, r, 1.0);\n"
    "    return fma(r, fma(err, err, err), r);\n"
    "  }\n"
    "  return tl_rcp_slow(d);\n}\n";

void generate(Program &P)
{
    // table layout: inputs then outputs, each tensor's stored components in storage order
    P.n_in = P.n_out = 0;
    std::ostringstream names;
    for (auto &t : P.tensors)
        if (t.kind == 0) {
            t.table_base = P.n_in;
            P.n_in += (int)t.stored.size();
        }
    for (auto &t : P.tensors)
        if (t.kind == 1) {
            t.table_base = P.n_out;
            P.n_out += (int)t.stored.size();
        }
    for (int pass = 0; pass < 2; ++pass)
        for (auto &t : P.tensors)
            if (t.kind == pass)
                for (auto &tup : t.stored) {
                    names << (pass == 0 ? "in " : "out ") << t.name;
                    for (int v : tup)
                        names << " " << v;
                    names << "\n";
                }
    P.names = names.str();
    if (P.n_out == 0)
        throw Error{"the program declares no output"};
    if (P.n_in + P.n_out > 480)
        throw Error{"more than 480 component arrays"};

    GenState G;
    G.defined.resize(P.tensors.size());
    // Each input is loaded just before the first statement that reads it (prefetched into L1 at the top
    // of the point when that statement is not the first to read inputs), and each output is stored
    // right after the last statement that assigns it: the registers an input or an output occupies are
    // held only while it is in use, as in the hand-written kernels.
    std::vector<int> last_def(P.tensors.size(), -1);
    for (size_t k = 0; k < P.stmts.size(); ++k)
        last_def[P.stmts[k].tensor] = (int)k;
    std::vector<std::pair<int, int>> in_of(P.n_in > 0 ? (size_t)P.n_in : 0);   // table position -> (tensor, slot)
    for (auto &t : P.tensors)
        if (t.kind == 0)
            for (size_t slot = 0; slot < t.stored.size(); ++slot)
                in_of[(size_t)(t.table_base + (int)slot)] = {(int)(&t - &P.tensors[0]), (int)slot};
    std::ostringstream body, prefetch;
    bool loaded_any = false;
    for (auto &st : P.stmts) {
        const Tensor &t = P.tensors[st.tensor];
        const int si = (int)(&st - &P.stmts[0]);
        std::ostringstream sb;
        G.body = &sb;
        const std::set<int> read_before = G.used_inputs;
        std::map<char, int> free_rhs;
        free_letters(P, *st.rhs, free_rhs, std::set<char>());
        std::set<char> lhs_letters;
        for (size_t s = 0; s < st.lhs.size(); ++s)
            if (!st.lhs[s].fixed) {
                if (st.lhs[s].value != 0)
                    throw Error{"offsets are not allowed on the left-hand side"};
                if (lhs_letters.count(st.lhs[s].letter))
                    throw Error{"left-hand side of '" + t.name + "' repeats an index"};
                lhs_letters.insert(st.lhs[s].letter);
            }
        std::set<char> rhs_letters;
        for (auto &kv : free_rhs)
            rhs_letters.insert(kv.first);
        if (rhs_letters != lhs_letters)
            throw Error{"free indices of the right-hand side differ from the left-hand side of '" + t.name + "'"};
        // every LHS index assignment whose tuple is a stored component
        std::vector<char> letters(lhs_letters.begin(), lhs_letters.end());
        std::vector<int> extent;
        for (char l : letters)
            for (size_t s = 0; s < st.lhs.size(); ++s)
                if (!st.lhs[s].fixed && st.lhs[s].letter == l) {
                    extent.push_back(range_of(P, l, t.dims[s]));
                    break;
                }
        std::vector<int> val(letters.size(), 0);
        std::vector<int> done_slots;
        for (;;) {
            Binding bind;
            for (size_t q = 0; q < letters.size(); ++q)
                bind[letters[q]] = val[q];
            std::vector<int> tup;
            for (auto &ix : st.lhs)
                tup.push_back(ix.fixed ? ix.value : bind[ix.letter]);
            bool in_range = true;
            for (size_t s = 0; s < tup.size(); ++s)
                in_range &= tup[s] >= 0 && tup[s] < t.dims[s];
            if (!in_range)
                throw Error{"fixed index out of range on the left-hand side of '" + t.name + "'"};
            const int slot = t.slot_of.at(tup);
            if (std::find(done_slots.begin(), done_slots.end(), slot) == done_slots.end()) {
                std::string rhs = gen(P, *st.rhs, bind, G);
                sb << "    const double " << value_name(P, st.tensor, slot) << "_s" << si << " = " << rhs << ";\n";
                done_slots.push_back(slot);
            }
            int r = (int)letters.size() - 1;
            while (r >= 0 && ++val[r] == extent[r])
                val[r--] = 0;
            if (r < 0)
                break;
        }
        // the inputs this statement reads first, loaded here; then its code
        std::vector<int> fresh;
        for (int q : G.used_inputs)
            if (!read_before.count(q))
                fresh.push_back(q);
        if (!fresh.empty()) {
            if (loaded_any)
                body << "    asm volatile(\"\" ::: \"memory\");   // not hoisted above the statements before\n";
            for (int q : fresh) {
                const auto ts = in_of[(size_t)q];
                body << "    const double " << value_name(P, ts.first, ts.second) << " = __ldcs(a.in[" << q << "] + x);\n";
                if (loaded_any)
                    prefetch << "    asm volatile(\"prefetch.global.L1 [%0];\" :: \"l\"(a.in[" << q << "] + x));\n";
            }
            if (!loaded_any)
                body << "    asm volatile(\"\" ::: \"memory\");   // issued before any arithmetic\n";
            loaded_any = true;
        }
        body << sb.str();
        // publish this statement's values under the tensor's component names; a component assigned a
        // second time invalidates the hoisted reciprocals and scaled factors (they may name it)
        for (int slot : done_slots)
            if (G.defined[st.tensor].count(slot)) {
                G.recip.clear();
                G.scaled.clear();
            }
        for (int slot : done_slots) {
            body << "    " << (G.defined[st.tensor].count(slot) ? "" : "double ") << value_name(P, st.tensor, slot)
                 << " = " << value_name(P, st.tensor, slot) << "_s" << &st - &P.stmts[0] << ";\n";
            G.defined[st.tensor].insert(slot);
        }
        if (t.kind == 1 && last_def[st.tensor] == si)
            for (size_t slot = 0; slot < t.stored.size(); ++slot)
                if (G.defined[st.tensor].count((int)slot))
                    body << "    __stcs(a.out[" << t.table_base + (int)slot << "] + x, "
                         << value_name(P, st.tensor, (int)slot) << ");\n";
    }
    G.body = nullptr;
    for (auto &t : P.tensors)
        if (t.kind == 1)
            for (size_t slot = 0; slot < t.stored.size(); ++slot)
                if (!G.defined[&t - &P.tensors[0]].count((int)slot))
                    throw Error{"output component " + std::to_string(slot) + " of '" + t.name + "' is never assigned"};

    std::ostringstream src;
    src << "// generated from a tensor-index program; one thread per grid point\n"
        << "// x * 2^k (|k| <= 8) by adjusting the exponent field with an integer add; zero, subnormal, huge,\n"
        << "// inf and nan operands take the multiplication, out of line: inline, the compiler if-converts it\n"
        << "// and every call then occupies an FP64 issue slot even with its predicate off\n"
        << "__device__ __noinline__ double tl_pow2_slow(double x, int k)\n{\n"
        << "  return x * __hiloint2double((1023 + k) << 20, 0);\n}\n"
        << "__device__ __forceinline__ double tl_pow2(double x, int k)\n{\n"
        << "  const int hi = __double2hiint(x), lo = __double2loint(x);\n"
        << "  const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;\n"
        << "  if (e > 8u && e < 2047u - 8u) { int r; asm(\"add.s32 %0, %1, %2;\" : \"=r\"(r) : \"r\"(hi), \"r\"(k << 20));\n"
        << "    return __hiloint2double(r, lo); }\n"
        << "  if (((hi & 0x7fffffff) | lo) == 0) return x;\n"
        << "  return tl_pow2_slow(x, k);\n}\n"
        << kMulSource
        << "struct TlJitArgs { const double *in[" << std::max(P.n_in, 1) << "]; double *out[" << P.n_out << "]; };\n"
        << "#ifndef TL_JIT_MIN_BLOCKS\n#define TL_JIT_MIN_BLOCKS 2\n#endif\n"
        << "extern \"C\" __global__ void __launch_bounds__(256, TL_JIT_MIN_BLOCKS) tl_jit_kernel(const TlJitArgs a, "
           "long long n)\n{\n"
        << "  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;\n"
        << "       x += (long long)gridDim.x * blockDim.x) {\n";
    src << prefetch.str() << body.str() << "  }\n}\n";
    P.source = src.str();
    P.reads.assign((size_t)P.n_in, 0);
    for (int q : G.used_inputs)
        P.reads[(size_t)q] = 1;
}

// ---------------------------------------------------------------------------------------------- NVRTC
typedef int (*nvrtcCreateProgram_t)(void **, const char *, const char *, int, const char *const *, const char *const *);
typedef int (*nvrtcCompileProgram_t)(void *, int, const char *const *);
typedef int (*nvrtcGetSize_t)(void *, size_t *);
typedef int (*nvrtcGetData_t)(void *, char *);
typedef int (*nvrtcDestroyProgram_t)(void **);

struct Nvrtc {
    bool tried = false, ok = false;
    nvrtcCreateProgram_t create = nullptr;
    nvrtcCompileProgram_t compile = nullptr;
    nvrtcGetSize_t log_size = nullptr, cubin_size = nullptr;
    nvrtcGetData_t log = nullptr, cubin = nullptr;
    nvrtcDestroyProgram_t destroy = nullptr;
};
Nvrtc g_nvrtc;
std::mutex g_nvrtc_mu;

bool load_nvrtc(std::string &why)
{
    std::lock_guard<std::mutex> lk(g_nvrtc_mu);
    if (!g_nvrtc.tried) {
        g_nvrtc.tried = true;
        const char *cands[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *c : cands)
            if ((h = dlopen(c, RTLD_NOW | RTLD_LOCAL)))
                break;
        if (h) {
            g_nvrtc.create = (nvrtcCreateProgram_t)dlsym(h, "nvrtcCreateProgram");
            g_nvrtc.compile = (nvrtcCompileProgram_t)dlsym(h, "nvrtcCompileProgram");
            g_nvrtc.log_size = (nvrtcGetSize_t)dlsym(h, "nvrtcGetProgramLogSize");
            g_nvrtc.log = (nvrtcGetData_t)dlsym(h, "nvrtcGetProgramLog");
            g_nvrtc.cubin_size = (nvrtcGetSize_t)dlsym(h, "nvrtcGetCUBINSize");
            g_nvrtc.cubin = (nvrtcGetData_t)dlsym(h, "nvrtcGetCUBIN");
            g_nvrtc.destroy = (nvrtcDestroyProgram_t)dlsym(h, "nvrtcDestroyProgram");
            g_nvrtc.ok = g_nvrtc.create && g_nvrtc.compile && g_nvrtc.log_size && g_nvrtc.log && g_nvrtc.cubin_size &&
                         g_nvrtc.cubin && g_nvrtc.destroy;
        }
    }
    if (!g_nvrtc.ok)
        why = "NVRTC (libnvrtc.so.13) could not be loaded";
    return g_nvrtc.ok;
}

// Compiled images by generated source (with the blocks per SM they were compiled for): programs that
// generate the same source compile once per process.
std::map<std::string, std::pair<std::vector<char>, int>> g_cubin_cache;
std::mutex g_cubin_mu;

bool nvrtc_compile_uncached(const std::string &src, std::vector<char> &cubin, std::string &log, int &min_blocks);

bool nvrtc_compile(const std::string &src, std::vector<char> &cubin, std::string &log, int &min_blocks)
{
    {
        std::lock_guard<std::mutex> lk(g_cubin_mu);
        auto it = g_cubin_cache.find(src);
        if (it != g_cubin_cache.end()) {
            cubin = it->second.first;
            min_blocks = it->second.second;
            return true;
        }
    }
    if (!nvrtc_compile_uncached(src, cubin, log, min_blocks))
        return false;
    std::lock_guard<std::mutex> lk(g_cubin_mu);
    g_cubin_cache.emplace(src, std::make_pair(cubin, min_blocks));
    return true;
}

void remember_cubin(const std::string &src, const std::vector<char> &cubin, int min_blocks)
{
    std::lock_guard<std::mutex> lk(g_cubin_mu);
    g_cubin_cache[src] = std::make_pair(cubin, min_blocks);
}

// Bytes of spill stores ptxas reports for tl_jit_kernel in a compile log (-1 when the log has none).
long spill_stores(const std::string &log)
{
    const size_t k = log.find("Function properties for tl_jit_kernel");
    if (k == std::string::npos)
        return -1;
    const size_t s = log.find("bytes spill stores", k);
    if (s == std::string::npos)
        return -1;
    size_t b = log.rfind(',', s);
    b = (b == std::string::npos || b < k) ? log.find('.', k) : b;
    return b == std::string::npos ? -1 : strtol(log.c_str() + b + 1, nullptr, 10);
}

bool nvrtc_compile_once(const std::string &src, int min_blocks, std::vector<char> &cubin, std::string &log);

// Three 256-thread blocks per SM (at most 85 registers) unless that spills more than 128 bytes per
// thread, then two (at most 128): a long chain such as Eq. 6 fits in 80 registers at three blocks
// and runs faster with the extra warps (3.03 -> 2.98 ms for the chain at N = 2^24), while the large
// contractions keep their registers.  The ptxas report in the compile log decides here when it is
// there; the first load on a device checks the kernel's local memory as well.
bool nvrtc_compile_uncached(const std::string &src, std::vector<char> &cubin, std::string &log, int &min_blocks)
{
    min_blocks = 3;
    if (!nvrtc_compile_once(src, min_blocks, cubin, log))
        return false;
    const long spills = spill_stores(log);
    if (spills <= 128)   // no report (-1): the first load on a device decides
        return true;
    min_blocks = 2;
    return nvrtc_compile_once(src, min_blocks, cubin, log);
}

bool nvrtc_compile_once(const std::string &src, int min_blocks, std::vector<char> &cubin, std::string &log)
{
    if (!load_nvrtc(log))
        return false;
    void *prog = nullptr;
    if (g_nvrtc.create(&prog, src.c_str(), "tl_jit.cu", 0, nullptr, nullptr) != 0) {
        log = "nvrtcCreateProgram failed";
        return false;
    }
    const std::string blocks = "-DTL_JIT_MIN_BLOCKS=" + std::to_string(min_blocks);
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", "--ptxas-options=-v",
                          blocks.c_str()};
    const int rc = g_nvrtc.compile(prog, 5, opts);
    size_t ls = 0;
    g_nvrtc.log_size(prog, &ls);
    log.assign(ls, '\0');
    if (ls)
        g_nvrtc.log(prog, &log[0]);
    while (!log.empty() && log.back() == '\0')   // the reported size counts the terminator
        log.pop_back();
    bool ok = rc == 0;
    if (ok) {
        size_t cs = 0;
        ok = g_nvrtc.cubin_size(prog, &cs) == 0 && cs > 0;
        if (ok) {
            cubin.resize(cs);
            ok = g_nvrtc.cubin(prog, cubin.data()) == 0;
        }
    }
    g_nvrtc.destroy(&prog);
    return ok;
}

}  // namespace jit
}  // namespace tl

struct tl_jit_kernel {
    uint64_t magic = 0;
    tl::jit::Program prog;
    std::vector<char> cubin;
    int min_blocks = 0;                         // the launch bound it was compiled for (blocks per SM)
    std::mutex mu;
    cudaLibrary_t lib[tl::kMaxDevices] = {};
    cudaKernel_t kern[tl::kMaxDevices] = {};
    int blocks[tl::kMaxDevices] = {};
};

using namespace tl;
static constexpr uint64_t kJitMagic = 0x746c5f6a69743031ull;

extern "C" {

tl_status tl_jit_compile(const char *program, tl_jit_kernel **out, char *log, size_t log_size)
{
    if (log && log_size)
        log[0] = '\0';
    if (!program || !out)
        return fail(TL_ERR_INVALID_ARG, "NULL program or output");
    *out = nullptr;
    auto k = std::make_unique<tl_jit_kernel>();
    std::string why;
    bool ok = false;
    try {
        const std::string text(program);   // the parser keeps a reference: it must outlive ps
        jit::Parser ps(text, k->prog);
        ps.parse();
        jit::generate(k->prog);
        ok = true;
    } catch (const jit::Error &e) {
        why = e.msg;
    }
    if (ok && !jit::nvrtc_compile(k->prog.source, k->cubin, why, k->min_blocks)) {
        ok = false;
        why = "NVRTC: " + why;
    }
    if (!ok) {
        if (log && log_size)
            snprintf(log, log_size, "%s", why.c_str());
        return fail(TL_ERR_INVALID_ARG, "%s", why.c_str());
    }
    k->magic = kJitMagic;
    *out = k.release();
    return TL_OK;
}

tl_status tl_jit_info(const tl_jit_kernel *k, int32_t *n_in, int32_t *n_out, const char **source,
                      const char **component_names)
{
    if (!k || k->magic != kJitMagic)
        return fail(TL_ERR_INVALID_ARG, "not a compiled program");
    if (n_in)
        *n_in = k->prog.n_in;
    if (n_out)
        *n_out = k->prog.n_out;
    if (source)
        *source = k->prog.source.c_str();
    if (component_names)
        *component_names = k->prog.names.c_str();
    return TL_OK;
}

tl_status tl_jit_reads(const tl_jit_kernel *k, uint8_t *reads)
{
    if (!k || k->magic != kJitMagic)
        return fail(TL_ERR_INVALID_ARG, "not a compiled program");
    if (!reads && k->prog.n_in)
        return fail(TL_ERR_INVALID_ARG, "NULL reads");
    for (int q = 0; q < k->prog.n_in; ++q)
        reads[q] = k->prog.reads[(size_t)q];
    return TL_OK;
}

tl_status tl_jit_launch(tl_jit_kernel *k, const double *const *in, double *const *out, int64_t n, tl_stream stream)
{
    if (!k || k->magic != kJitMagic)
        return fail(TL_ERR_INVALID_ARG, "not a compiled program");
    if ((k->prog.n_in && !in) || !out)
        return fail(TL_ERR_INVALID_ARG, "NULL table");
    if (n < 0)
        return fail(TL_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    const void *const *tabs[2] = {(const void *const *)in, (const void *const *)out};
    const int counts[2] = {k->prog.n_in, k->prog.n_out};
    const bool writes[2] = {false, true}, nullable[2] = {false, false};
    const char *const names[2] = {"in", "out"};
    std::vector<Range> rs;
    tl_status s = collect_ranges(rs, tabs, counts, writes, nullable, names, 2, n, sizeof(double), -1);
    if (s == TL_OK)
        s = check_overlaps(rs);
    if (s != TL_OK || n == 0)
        return s;
    const DeviceInfo *d = nullptr;
    if ((s = device_info(&d)) != TL_OK)
        return s;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e;
    {
        std::lock_guard<std::mutex> lk(k->mu);
        if (!k->kern[dev]) {   // load the module on this device once
            if ((e = cudaLibraryLoadData(&k->lib[dev], k->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0)) !=
                cudaSuccess)
                return cuda_fail(e, "cudaLibraryLoadData");
            if ((e = cudaLibraryGetKernel(&k->kern[dev], k->lib[dev], "tl_jit_kernel")) != cudaSuccess)
                return cuda_fail(e, "cudaLibraryGetKernel");
            if (k->min_blocks == 3) {
                // The loaded kernel's local memory decides (the compile log carries no ptxas report
                // under some tools, e.g. a profiler): more than 128 bytes per thread at three blocks
                // per SM, and it is rebuilt for two.
                cudaFuncAttributes fa;
                if ((e = cudaFuncGetAttributes(&fa, (const void *)k->kern[dev])) != cudaSuccess)
                    return cuda_fail(e, "cudaFuncGetAttributes");
                if (fa.localSizeBytes > 128) {
                    std::vector<char> cubin;
                    std::string why;
                    if (!jit::nvrtc_compile_once(k->prog.source, 2, cubin, why))
                        return fail(TL_ERR_INVALID_ARG, "NVRTC: %s", why.c_str());
                    cudaLibraryUnload(k->lib[dev]);
                    k->lib[dev] = nullptr;
                    k->kern[dev] = nullptr;
                    k->cubin.swap(cubin);
                    k->min_blocks = 2;
                    jit::remember_cubin(k->prog.source, k->cubin, 2);
                    if ((e = cudaLibraryLoadData(&k->lib[dev], k->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr,
                                                 0)) != cudaSuccess)
                        return cuda_fail(e, "cudaLibraryLoadData");
                    if ((e = cudaLibraryGetKernel(&k->kern[dev], k->lib[dev], "tl_jit_kernel")) != cudaSuccess)
                        return cuda_fail(e, "cudaLibraryGetKernel");
                }
            }
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k->blocks[dev], (const void *)k->kern[dev], 256, 0)) !=
                cudaSuccess)
                return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        }
    }
    std::vector<const void *> argbuf((size_t)std::max(k->prog.n_in, 1) + k->prog.n_out, nullptr);
    for (int q = 0; q < k->prog.n_in; ++q)
        argbuf[q] = in[q];
    for (int q = 0; q < k->prog.n_out; ++q)
        argbuf[std::max(k->prog.n_in, 1) + q] = out[q];
    long long nn = (long long)n;
    void *args[2] = {argbuf.data(), &nn};
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)d->sms * std::max(1, k->blocks[dev])));
    if ((e = cudaLaunchKernel((const void *)k->kern[dev], dim3(grid), dim3(256), args, 0, (cudaStream_t)stream)) !=
        cudaSuccess)
        return cuda_fail(e, "generated kernel launch");
    return TL_OK;
}

void tl_jit_destroy(tl_jit_kernel *k)
{
    if (!k || k->magic != kJitMagic)
        return;
    for (int dv = 0; dv < kMaxDevices; ++dv)
        if (k->lib[dv])
            cudaLibraryUnload(k->lib[dv]);
    k->magic = 0;
    delete k;
}

}  // extern "C"

extern "C" TL_API tl_status tl_testing_jit_min_blocks(const tl_jit_kernel *k, int32_t *blocks)
{
    if (!k || k->magic != kJitMagic || !blocks)
        return TL_ERR_INVALID_ARG;
    *blocks = k->min_blocks;
    return TL_OK;
}
