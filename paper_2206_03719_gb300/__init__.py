"""GB300-native Heston / Longstaff-Schwartz / bump-and-revalue Greeks."""
