"""CPU tests of libmk's large-frame host side: the stress templates and the
adversarial relation generators (mk_template, mk_stress_relation) against
the oracle's independent constructions, bit for bit; the config struct and
the key packing.  No GPU and no kernel is called here."""
import ctypes

import pytest

import oracle
from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()


def test_stress_cfg_layout():
    assert ctypes.sizeof(mk.mk_stress_cfg) == 32
    assert mk.relation_words(16, 33) == 2 * 256 and mk.relation_words(6, 32) == 36
    assert mk.relation_words(0, 10) == 0 and mk.relation_words(17, 10) == 0


@pytest.mark.parametrize("n", (1, 2, 3, 6, 8, 11, 16))
def test_templates_match_oracle(n):
    for t in range(mk.NUM_TEMPLATES):
        assert mk.template(t, n) == oracle.template(t, n), (t, n)


@pytest.mark.parametrize("gen", mk.GENERATORS)
@pytest.mark.parametrize("n", (2, 5, 6, 8, 9, 12, 16))
def test_generators_match_oracle(gen, n):
    for s in list(range(200)) + [10 ** 6, 2 ** 40 + 3]:
        assert mk.stress_relation(gen, 1234, n, s) == oracle.stress_relation(gen, 1234, n, s), (gen, n, s)


def test_erdos_renyi_small_sizes_are_the_sampled_family():
    for n in (1, 4, 7, 8):
        for s in range(50):
            m = mk.sample_relation(9, n, s)
            assert mk.stress_relation("er", 9, n, s) == [(m >> (w * n)) & ((1 << n) - 1) for w in range(n)]


def test_invalid_arguments_rejected():
    with pytest.raises(mk.MkError):
        mk.template(39, 6)
    with pytest.raises(mk.MkError):
        mk.template(0, 17)
    with pytest.raises(mk.MkError):
        mk.stress_relation("scc", 1, 1, 0)       # two blocks need two worlds
    with pytest.raises(mk.MkError):
        mk.stress_relation(6, 1, 8, 0)


def test_key_decoding():
    key = (123456 << 20) | (4095 << 4) | 11
    assert mk.decode_stress_key(key) == (123456, 4095, 11)
    assert mk.decode_stress_key(mk.NO_KEY) is None
