"""Host-side policy of the driver (no GPU): which exact assignment form a dimension gets."""
from paper_1502_04265_gb300 import driver


def test_exact_form_threshold():
    assert driver.exact_form(1) == "f32"
    assert driver.exact_form(64) == "f32"
    assert driver.exact_form(driver.BF16_MIN_D - 1) == "f32"
    assert driver.exact_form(driver.BF16_MIN_D) == "bf16"
    assert driver.exact_form(1024) == "bf16"
    assert driver.exact_form(1030) == "f32"   # BF16 tcgen05 operands need d % 8 == 0
