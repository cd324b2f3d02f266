"""Each plausible mistake in the oracle (an off-by-one predicate, the wrong
hash bits, a dropped or sign-flipped term, a reversed tie-break, a wrong join
index, transposed operands, and in the aggregate-first plan a semi-join
taken as a join, a non-strict threshold, a dropped D' or date filter) must
trip at least one pin.

The shipped oracle holds no switch for these mistakes: each mutant is a copy
of oracle.cpp with one line replaced, compiled into a library of its own
under the test's temporary directory and swapped in only for the duration of
the pins."""
import os
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.cpp")

# (name, text of the oracle, the same text with the mistake)
MUTANTS = [
    ("'<' evaluated as '<='", "case 0: return v < c;", "case 0: return v <= c;"),
    ("partition on the low hash bits", "return h >> (64 - log2P);",
     "return h & ((1ULL << log2P) - 1);"),
    ("revenue drops the (100 - disc) factor",
     "const __int128 revenue = static_cast<__int128>(f_price[i]) * (100 - f_disc[i]);",
     "const __int128 revenue = static_cast<__int128>(f_price[i]);"),
    ("revenue uses (100 + disc)",
     "const __int128 revenue = static_cast<__int128>(f_price[i]) * (100 - f_disc[i]);",
     "const __int128 revenue = static_cast<__int128>(f_price[i]) * (100 + f_disc[i]);"),
    ("top-k tie-break on key descending", "return ka < kb;", "return ka > kb;"),
    ("M.dref looked up off by one", "const int64_t ref = m_dref[i];",
     "const int64_t ref = int64_t{m_dref[i]} + 1;"),
    ("group-by with key and value transposed", "groups[load(key, ktype, i)] += val[i];",
     "groups[val[i]] += load(key, ktype, i);"),
    ("join pair with probe row and build value swapped", "pairs.emplace_back(i, it->second);",
     "pairs.emplace_back(it->second, i);"),
    ("aggregate-first semi-join counts a key once per M' row", "const __int128 sum = kv.second;",
     "const __int128 sum = m != m_keys.end() ? kv.second * m->second : kv.second;"),
    ("aggregate-first threshold compared with >=", "if (sum > having && m != m_keys.end())",
     "if (sum >= having && m != m_keys.end())"),
    ("aggregate-first M' ignores D'",
     "if (pred(m_op, m_date[i], m_c) && d_pass.count(m_dref[i])) ++m_keys[m_key[i]];",
     "if (pred(m_op, m_date[i], m_c)) ++m_keys[m_key[i]];"),
    ("aggregate-first aggregation drops the F date filter",
     "if (pred(f_op, f_date2[i], f_c))\n      g[f_mkey[i]]", "if (true)\n      g[f_mkey[i]]"),
]


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, orig, bad):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"the oracle line of mutant '{name}' is not unique"
    src = tmp_path / "mutant.cpp"
    src.write_text(text.replace(orig, bad))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-o", str(lib), str(src)],
                   check=True)
    failures = []
    with oracle.variant(str(lib)):
        for pin in pins.ALL_PINS:
            try:
                pin()
            except AssertionError:
                failures.append(pin.__name__)
    assert failures, f"mutant '{name}' passed every pin"
